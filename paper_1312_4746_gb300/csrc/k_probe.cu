// Issue rates of the arithmetic pipes that the pixel x sample sums lean on,
// measured on the device: sustained results per SM per clock of the
// exponential (ex2.approx, the special-function unit), popc, FFMA and the
// packed FFMA2 (fma.rn.f32x2, two results per instruction). These are the
// denominators of the sums' ALU rooflines; nothing of the method runs here.
//
// One block of 1024 threads per SM (the dynamic shared-memory request keeps
// a second block off the SM); every thread runs 8 independent chains of the
// probed operation, so 64 chains per scheduler cover the pipes' latencies.
// Each block reads its SM's cycle counter around the loop after a block
// barrier; the rate of a block is its results / its cycles (clock cycles of
// its own SM, so the figure is per clock whatever the clock frequency was).
#include <algorithm>
#include <cstdint>
#include <vector>

#include "internal.h"

namespace {

constexpr int PT = 1024;                // threads per probe block
constexpr int CH = 8;                   // independent chains per thread
constexpr int PROBE_SMEM = 120 * 1024;  // more than half of an SM's shared memory

enum ProbeOp { OP_EX2 = 0, OP_POPC = 1, OP_FFMA = 2, OP_FFMA2 = 3 };

__device__ __forceinline__ float ex2_neg(float x) {
    float y;
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(-x));
    return y;  // x in (0, 1] stays in [0.5, 1)
}

__device__ __forceinline__ uint64_t ffma2(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t d;
    asm volatile("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

template <int OP>
__global__ void __launch_bounds__(PT, 1) probe_kernel(int iters, long long* cycles,
                                                      unsigned* sink) {
    extern __shared__ unsigned char probe_smem[];  // occupancy only
    const unsigned tid = threadIdx.x;
    float f[CH];
    unsigned u[CH];
    uint64_t p[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) {
        f[c] = 0.25f + 0.01f * (float)((tid + c) & 63);
        u[c] = tid * 2654435761u + (unsigned)c;
        p[c] = ((uint64_t)__float_as_uint(f[c] + 0.5f) << 32) | __float_as_uint(f[c]);
    }
    const float a = 0.999f, b = 0.001f;
    const uint64_t a2 = ((uint64_t)__float_as_uint(a) << 32) | __float_as_uint(a);
    const uint64_t b2 = ((uint64_t)__float_as_uint(b) << 32) | __float_as_uint(b);
    __syncthreads();
    const long long t0 = clock64();
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            if (OP == OP_EX2) f[c] = ex2_neg(f[c]);
            if (OP == OP_POPC) u[c] = __popc(u[c]);
            if (OP == OP_FFMA) f[c] = fmaf(f[c], a, b);
            if (OP == OP_FFMA2) p[c] = ffma2(p[c], a2, b2);
        }
    }
    __syncthreads();
    const long long t1 = clock64();
    unsigned acc = 0;
#pragma unroll
    for (int c = 0; c < CH; ++c)
        acc ^= __float_as_uint(f[c]) ^ u[c] ^ (unsigned)p[c] ^ (unsigned)(p[c] >> 32);
    sink[blockIdx.x * PT + tid] = acc;  // keeps every chain live
    if (tid == 0) cycles[blockIdx.x] = t1 - t0;
    if (tid == 0 && iters < 0) probe_smem[0] = 0;
}

template <int OP>
cudaError_t run_probe(int n_sm, int iters, long long* d_cycles, unsigned* d_sink,
                      std::vector<long long>& cyc, float* ms) {
    cudaError_t e = cudaFuncSetAttribute(probe_kernel<OP>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, PROBE_SMEM);
    cudaEvent_t ev[2] = {nullptr, nullptr};
    if (e == cudaSuccess) e = cudaEventCreate(&ev[0]);
    if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {  // the first launch warms up
        if (rep == 1) e = cudaEventRecord(ev[0]);
        if (e == cudaSuccess) {
            probe_kernel<OP><<<n_sm, PT, PROBE_SMEM>>>(iters, d_cycles, d_sink);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess && rep == 1) e = cudaEventRecord(ev[1]);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
    }
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, ev[0], ev[1]);
    for (cudaEvent_t x : ev)
        if (x) cudaEventDestroy(x);
    if (e != cudaSuccess) return e;
    cyc.resize(n_sm);
    return cudaMemcpy(cyc.data(), d_cycles, sizeof(long long) * n_sm, cudaMemcpyDeviceToHost);
}

}  // namespace

extern "C" cs_status cs_unit_rates(cs_ctx* ctx, double* out, double* clock_mhz) {
    const char* fn = "cs_unit_rates";
    if (!ctx) return cs_set_error(nullptr, CS_ERR_INVALID_ARG, "%s: ctx is NULL", fn);
    if (!out) return cs_set_error(ctx, CS_ERR_INVALID_ARG, "%s: out is NULL", fn);
    DeviceGuard g(ctx->device);
    const int n_sm = ctx->n_sm;
    long long* d_cycles = nullptr;
    unsigned* d_sink = nullptr;
    cudaError_t e = cudaMalloc(&d_cycles, sizeof(long long) * n_sm);
    if (e == cudaSuccess) e = cudaMalloc(&d_sink, sizeof(unsigned) * (size_t)n_sm * PT);
    // iterations per op: about a millisecond each at the nominal rates
    const int iters[4] = {2048, 2048, 8192, 4096};
    const double per_iter[4] = {CH, CH, CH, 2.0 * CH};  // results per thread per iteration
    double clk = 0.0;
    for (int op = 0; op < 4 && e == cudaSuccess; ++op) {
        std::vector<long long> cyc;
        float ms = 0.f;
        switch (op) {
            case OP_EX2: e = run_probe<OP_EX2>(n_sm, iters[op], d_cycles, d_sink, cyc, &ms); break;
            case OP_POPC: e = run_probe<OP_POPC>(n_sm, iters[op], d_cycles, d_sink, cyc, &ms); break;
            case OP_FFMA: e = run_probe<OP_FFMA>(n_sm, iters[op], d_cycles, d_sink, cyc, &ms); break;
            default: e = run_probe<OP_FFMA2>(n_sm, iters[op], d_cycles, d_sink, cyc, &ms); break;
        }
        if (e != cudaSuccess) break;
        std::sort(cyc.begin(), cyc.end());
        const double med = (double)cyc[cyc.size() / 2];
        out[op] = (double)PT * iters[op] * per_iter[op] / med;
        // the SM clock implied by the longest block's cycles over the launch time
        if (op == OP_FFMA && ms > 0.f) clk = (double)cyc.back() / (ms * 1e3);
    }
    if (d_cycles) cudaFree(d_cycles);
    if (d_sink) cudaFree(d_sink);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cs_set_error(ctx, CS_ERR_CUDA, "%s: %s", fn, cudaGetErrorString(e));
    }
    if (clock_mhz) *clock_mhz = clk;
    return CS_OK;
}
