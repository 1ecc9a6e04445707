// probe.cu -- diagnostics: per-SM issue rates of the FP32 pipe and of the MUFU ex2 unit
// (the two pipes that bound the render kernels), and an elementwise view of the
// exponential the render kernels use.
#include <algorithm>
#include <vector>

#include "bgs_internal.cuh"

namespace {

constexpr int kProbeThreads = 512;
constexpr int kProbeIters = 4096;

__device__ __forceinline__ unsigned smid() {
    unsigned r;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(r));
    return r;
}

// 8 independent FMA chains per thread; records (SM id, start clock, end clock) per block.
__global__ void __launch_bounds__(kProbeThreads) k_probe_fma(float seed, float *sink, long long *cycles) {
    float v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = seed + threadIdx.x * 1e-3f + k;
    __syncthreads();
    const long long t0 = clock64();
    for (int i = 0; i < kProbeIters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) asm volatile("fma.rn.f32 %0, %0, 0f3F7FBE77, 0f3A83126F;" : "+f"(v[k]));
    }
    __syncthreads();
    const long long t1 = clock64();
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += v[k];
    if (s == 12345.f) sink[threadIdx.x] = s;
    if (threadIdx.x == 0) {
        cycles[3 * blockIdx.x] = smid();
        cycles[3 * blockIdx.x + 1] = t0;
        cycles[3 * blockIdx.x + 2] = t1;
    }
}

// 8 independent ex2 chains per thread (the value is kept in a bounded range).
__global__ void __launch_bounds__(kProbeThreads) k_probe_ex2(float seed, float *sink, long long *cycles) {
    float v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = -(seed + threadIdx.x * 1e-4f + k * 0.01f);
    __syncthreads();
    const long long t0 = clock64();
    for (int i = 0; i < kProbeIters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) asm volatile("ex2.approx.ftz.f32 %0, %0;" : "+f"(v[k]));
    }
    __syncthreads();
    const long long t1 = clock64();
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += v[k];
    if (s == 12345.f) sink[threadIdx.x] = s;
    if (threadIdx.x == 0) {
        cycles[3 * blockIdx.x] = smid();
        cycles[3 * blockIdx.x + 1] = t0;
        cycles[3 * blockIdx.x + 2] = t1;
    }
}

__global__ void k_exp2(const float *x, float *y, long long n) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = bgs::ex2_approx(x[i]);
}

}  // namespace

extern "C" int bgs_probe_pipe_rates(bgs_plan *plan, double *fp32_per_sm_clk, double *ex2_per_sm_clk, void *stream) {
    if (!plan || !fp32_per_sm_clk || !ex2_per_sm_clk) return BGS_ERR_INVALID;
    const int sms = bgs_plan_num_sms(plan);
    cudaStream_t s = (cudaStream_t)stream;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_probe_fma, kProbeThreads, 0) != cudaSuccess)
        return BGS_ERR_CUDA;
    per_sm = std::max(1, std::min(per_sm, 4));
    const int blocks = sms * per_sm;
    float *sink = nullptr;
    long long *cyc = nullptr;
    if (cudaMalloc(&sink, sizeof(float) * kProbeThreads) != cudaSuccess) return BGS_ERR_CUDA;
    if (cudaMalloc(&cyc, sizeof(long long) * 3 * blocks) != cudaSuccess) {
        cudaFree(sink);
        return BGS_ERR_CUDA;
    }
    std::vector<long long> h(3 * blocks);
    double rates[2] = {0, 0};
    for (int which = 0; which < 2; ++which) {
        for (int rep = 0; rep < 2; ++rep) {  // first repetition warms up
            if (which == 0)
                k_probe_fma<<<blocks, kProbeThreads, 0, s>>>(1.0f, sink, cyc);
            else
                k_probe_ex2<<<blocks, kProbeThreads, 0, s>>>(0.5f, sink, cyc);
        }
        if (cudaMemcpyAsync(h.data(), cyc, sizeof(long long) * 3 * blocks, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            cudaFree(sink);
            cudaFree(cyc);
            return BGS_ERR_CUDA;
        }
        // per SM: operations of the blocks it ran / (last end - first start) on its clock
        const int max_sm = 1024;
        std::vector<long long> first(max_sm, -1), last(max_sm, -1), nblk(max_sm, 0);
        for (int b = 0; b < blocks; ++b) {
            const int id = (int)h[3 * b];
            if (id < 0 || id >= max_sm) continue;
            if (first[id] < 0 || h[3 * b + 1] < first[id]) first[id] = h[3 * b + 1];
            if (last[id] < 0 || h[3 * b + 2] > last[id]) last[id] = h[3 * b + 2];
            nblk[id] += 1;
        }
        std::vector<double> r;
        const double ops_per_block = (double)kProbeThreads * kProbeIters * 8;
        for (int id = 0; id < max_sm; ++id)
            if (nblk[id] > 0 && last[id] > first[id]) r.push_back(ops_per_block * nblk[id] / (double)(last[id] - first[id]));
        if (r.empty()) {
            cudaFree(sink);
            cudaFree(cyc);
            return BGS_ERR_CUDA;
        }
        std::sort(r.begin(), r.end());
        rates[which] = r[r.size() / 2];  // median over SMs
    }
    cudaFree(sink);
    cudaFree(cyc);
    *fp32_per_sm_clk = rates[0];
    *ex2_per_sm_clk = rates[1];
    return BGS_OK;
}

extern "C" int bgs_debug_exp2(const float *x, float *y, int64_t n, void *stream) {
    if (n < 0 || (n > 0 && (!x || !y))) return BGS_ERR_INVALID;
    if (n == 0) return BGS_OK;
    k_exp2<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(x, y, n);
    return cudaGetLastError() == cudaSuccess ? BGS_OK : BGS_ERR_CUDA;
}
