// Unsupervised mode (Sec. 3.2, "Unsupervised Segmentation"): k-means on the
// colour pixels, k-medians on the smooth co-supports iota(O s_x) of Eq.
// (map_tsm), segments = (colour class, texture class) pairs, each pixel's
// colour and texture likelihood as in Eq. (post_text).
//
// Both clusterings start from caller-given pixels and run a fixed number of
// rounds (assignment, then update), then a last assignment to the final
// centres. Assignments are decided in FP32 with the distances accumulated in
// a fixed order (colour ((d0^2 + d1^2) + d2^2), texture over codes
// j = 0 .. k-1), ties to the lower class, so they are reproducible bit for
// bit. A k-means centroid is the exact mean of the members' values rounded
// to multiples of 2^-24: integer sums (order-free atomics), one double
// division, one rounding to FP32. A k-medians centre is the elementwise
// median by radix selection over the class's member list. A class without
// members keeps its centre.
#include <cstdint>

#include "internal.h"

namespace {

constexpr int UB = 256;             // threads per block
constexpr float QSCALE = 16777216.f;  // 2^24

__global__ void kmeans_init_kernel(const float* __restrict__ X, UnsupInit init, int n,
                                   float* __restrict__ C) {
    const int t = threadIdx.x;
    if (t < 3 * n) C[t] = X[(size_t)init.v[t / 3] * 3 + t % 3];
}

__device__ __forceinline__ int nearest_colour(const float* x, const float* C, int n) {
    int best = 0;
    float bd = 0.f;
    for (int a = 0; a < n; ++a) {
        const float t0 = __fsub_rn(x[0], C[3 * a]);
        const float t1 = __fsub_rn(x[1], C[3 * a + 1]);
        const float t2 = __fsub_rn(x[2], C[3 * a + 2]);
        const float d =
            __fadd_rn(__fadd_rn(__fmul_rn(t0, t0), __fmul_rn(t1, t1)), __fmul_rn(t2, t2));
        if (a == 0 || d < bd) {
            bd = d;
            best = a;
        }
    }
    return best;
}

// Assignment to the nearest centre; with sums != null also the members'
// fixed-point sums and counts (per block in shared memory, then atomics).
__global__ void __launch_bounds__(UB) kmeans_assign_kernel(
    const float* __restrict__ X, int N, const float* __restrict__ Cg, int n,
    int32_t* __restrict__ assign, unsigned long long* __restrict__ sums,
    unsigned* __restrict__ counts) {
    __shared__ float C[3 * CS_MAX_CLASSES];
    __shared__ unsigned long long s_sum[3 * CS_MAX_CLASSES];
    __shared__ unsigned s_cnt[CS_MAX_CLASSES];
    for (int t = threadIdx.x; t < 3 * n; t += UB) {
        C[t] = Cg[t];
        s_sum[t] = 0ull;
    }
    for (int t = threadIdx.x; t < n; t += UB) s_cnt[t] = 0u;
    __syncthreads();
    for (int q = blockIdx.x * UB + threadIdx.x; q < N; q += gridDim.x * UB) {
        const float x[3] = {X[(size_t)q * 3], X[(size_t)q * 3 + 1], X[(size_t)q * 3 + 2]};
        const int a = nearest_colour(x, C, n);
        if (assign) assign[q] = a;
        if (sums) {
            for (int c = 0; c < 3; ++c)
                atomicAdd(s_sum + 3 * a + c,
                          (unsigned long long)__float2ll_rn(__fmul_rn(x[c], QSCALE)));
            atomicAdd(s_cnt + a, 1u);
        }
    }
    if (!sums) return;
    __syncthreads();
    for (int t = threadIdx.x; t < 3 * n; t += UB)
        if (s_sum[t]) atomicAdd(sums + t, s_sum[t]);
    for (int t = threadIdx.x; t < n; t += UB)
        if (s_cnt[t]) atomicAdd(counts + t, s_cnt[t]);
}

// C = float(S / (cnt 2^24)) for classes with members; clears the sums.
__global__ void kmeans_update_kernel(float* __restrict__ C, unsigned long long* __restrict__ sums,
                                     unsigned* __restrict__ counts, int n) {
    const int t = threadIdx.x;
    if (t < 3 * n) {
        const unsigned cnt = counts[t / 3];
        if (cnt) C[t] = (float)((double)(long long)sums[t] / ((double)cnt * 16777216.0));
    }
    __syncthreads();
    if (t < 3 * n) sums[t] = 0ull;
    if (t < n) counts[t] = 0u;
}

__global__ void kmedians_init_kernel(const float* __restrict__ V, int N, int k, UnsupInit init,
                                     int n, float* __restrict__ C) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n * k; t += gridDim.x * blockDim.x)
        C[t] = V[(size_t)(t % k) * N + init.v[t / k]];
}

// l1 distances of pixel q's column of V to the n centres in shared memory,
// summed over codes j = 0 .. k-1 in turn (FP32, no contraction).
__device__ __forceinline__ void l1_all(const float* __restrict__ V, int N, int k, int q,
                                       const float* C, int n, float (&d)[CS_MAX_CLASSES]) {
#pragma unroll
    for (int b = 0; b < CS_MAX_CLASSES; ++b) d[b] = 0.f;
    for (int j = 0; j < k; ++j) {
        const float v = V[(size_t)j * N + q];
#pragma unroll
        for (int b = 0; b < CS_MAX_CLASSES; ++b)
            if (b < n) d[b] = __fadd_rn(d[b], fabsf(__fsub_rn(C[b * k + j], v)));
    }
}

__global__ void __launch_bounds__(UB) kmedians_assign_kernel(
    const float* __restrict__ V, int N, int k, const float* __restrict__ Cg, int n,
    int32_t* __restrict__ assign, unsigned* __restrict__ counts) {
    extern __shared__ float C[];  // n x k
    __shared__ unsigned s_cnt[CS_MAX_CLASSES];
    for (int t = threadIdx.x; t < n * k; t += UB) C[t] = Cg[t];
    for (int t = threadIdx.x; t < n; t += UB) s_cnt[t] = 0u;
    __syncthreads();
    for (int q = blockIdx.x * UB + threadIdx.x; q < N; q += gridDim.x * UB) {
        float d[CS_MAX_CLASSES];
        l1_all(V, N, k, q, C, n, d);
        int best = 0;
#pragma unroll
        for (int b = 1; b < CS_MAX_CLASSES; ++b)
            if (b < n && d[b] < d[best]) best = b;
        assign[q] = best;
        if (counts) atomicAdd(s_cnt + best, 1u);
    }
    if (!counts) return;
    __syncthreads();
    for (int t = threadIdx.x; t < n; t += UB)
        if (s_cnt[t]) atomicAdd(counts + t, s_cnt[t]);
}

// Class offsets (exclusive scan of the counts), fill cursors cleared.
__global__ void class_offsets_kernel(unsigned* __restrict__ counts, int n,
                                     int32_t* __restrict__ off, unsigned* __restrict__ cursor) {
    if (threadIdx.x != 0) return;
    int acc = 0;
    for (int b = 0; b < n; ++b) {
        off[b] = acc;
        acc += (int)counts[b];
        counts[b] = 0u;
        cursor[b] = 0u;
    }
    off[n] = acc;
}

// Member lists by class (order within a class is free: medians do not see it).
__global__ void class_scatter_kernel(const int32_t* __restrict__ assign, int N,
                                     const int32_t* __restrict__ off, unsigned* __restrict__ cursor,
                                     int32_t* __restrict__ members) {
    const unsigned lane = threadIdx.x & 31u;
    for (int q = blockIdx.x * UB + threadIdx.x; q < N; q += gridDim.x * UB) {
        const int b = assign[q];
        // one atomic per class and warp: the lowest lane of each class group
        // reserves the group's slots
        const unsigned act = __activemask();
        const unsigned peers = __match_any_sync(act, b);
        const int leader = __ffs(peers) - 1;
        unsigned base = 0;
        if ((int)lane == leader) base = atomicAdd(cursor + b, (unsigned)__popc(peers));
        base = __shfl_sync(peers, base, leader);
        members[off[b] + (int)(base + __popc(peers & ((1u << lane) - 1u)))] = q;
    }
}

// Last step: colour and texture assignments to the final centres and the
// data term f_{a n_t + b} = -log P_colour(a) - log P_texture(b), each a
// softmax over its classes: logits -|I - mu_a|^2 / (2 sigma_c2) and
// -||c_b - iota||_1 / beta.
__global__ void __launch_bounds__(UB) unsup_final_kernel(
    const float* __restrict__ img, int P, const float* __restrict__ V, int k,
    const float* __restrict__ Ccol, int nc, const float* __restrict__ Ctex, int nt,
    float inv2s2, float inv_beta, float* __restrict__ neglog, int32_t* __restrict__ cassign,
    int32_t* __restrict__ tassign) {
    extern __shared__ float C[];  // nt x k texture centres
    __shared__ float Cc[3 * CS_MAX_CLASSES];
    for (int t = threadIdx.x; t < nt * k; t += UB) C[t] = Ctex[t];
    for (int t = threadIdx.x; t < 3 * nc; t += UB) Cc[t] = Ccol[t];
    __syncthreads();
    for (int q = blockIdx.x * UB + threadIdx.x; q < P; q += gridDim.x * UB) {
        const float x[3] = {img[(size_t)q * 3], img[(size_t)q * 3 + 1], img[(size_t)q * 3 + 2]};
        if (cassign) cassign[q] = nearest_colour(x, Cc, nc);
        float d[CS_MAX_CLASSES];
        l1_all(V, P, k, q, C, nt, d);
        int best = 0;
#pragma unroll
        for (int b = 1; b < CS_MAX_CLASSES; ++b)
            if (b < nt && d[b] < d[best]) best = b;
        if (tassign) tassign[q] = best;
        // texture log-softmax
        float tmax = -d[best] * inv_beta, ts = 0.f;
#pragma unroll
        for (int b = 0; b < CS_MAX_CLASSES; ++b)
            if (b < nt) ts += __expf(-d[b] * inv_beta - tmax);
        const float tlse = tmax + __logf(ts);
        // colour log-softmax
        float lc[CS_MAX_CLASSES];
        float cmax = -3.0e38f;
#pragma unroll
        for (int a = 0; a < CS_MAX_CLASSES; ++a)
            if (a < nc) {
                const float t0 = x[0] - Cc[3 * a], t1 = x[1] - Cc[3 * a + 1],
                            t2 = x[2] - Cc[3 * a + 2];
                lc[a] = -(t0 * t0 + t1 * t1 + t2 * t2) * inv2s2;
                cmax = fmaxf(cmax, lc[a]);
            }
        float cs = 0.f;
#pragma unroll
        for (int a = 0; a < CS_MAX_CLASSES; ++a)
            if (a < nc) cs += __expf(lc[a] - cmax);
        const float clse = cmax + __logf(cs);
        float ft[CS_MAX_CLASSES];
#pragma unroll
        for (int b = 0; b < CS_MAX_CLASSES; ++b) ft[b] = tlse + d[b] * inv_beta;
#pragma unroll 1
        for (int a = 0; a < nc; ++a) {
            const float fc = clse - lc[a];
#pragma unroll 1
            for (int b = 0; b < nt; ++b) neglog[(size_t)(a * nt + b) * P + q] = fc + ft[b];
        }
    }
}

int grid_for(long long N, int n_sm) {
    const long long need = (N + UB - 1) / UB, cap = 8ll * n_sm;
    return (int)(need < 1 ? 1 : need < cap ? need : cap);
}

cudaError_t set_smem(const void* f, size_t bytes) {
    return bytes > 48 * 1024
               ? cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes)
               : cudaSuccess;
}

}  // namespace

size_t kmeans_scratch_bytes(int n) {
    return sizeof(unsigned long long) * 3 * (size_t)n + sizeof(unsigned) * (size_t)n + 256;
}

size_t kmedians_scratch_bytes(long long N, int n) {
    return sizeof(int32_t) * ((size_t)N + (size_t)n + 1) + 2 * sizeof(unsigned) * (size_t)n + 256;
}

cudaError_t launch_kmeans(const KmeansArgs& a, cudaStream_t st) {
    unsigned long long* sums = reinterpret_cast<unsigned long long*>(a.scratch);
    unsigned* counts = reinterpret_cast<unsigned*>(sums + 3 * a.n);
    cudaError_t e = cudaMemsetAsync(a.scratch, 0, kmeans_scratch_bytes(a.n), st);
    if (e != cudaSuccess) return e;
    kmeans_init_kernel<<<1, 3 * CS_MAX_CLASSES, 0, st>>>(a.X, a.init, a.n, a.C);
    const int g = grid_for(a.N, a.n_sm);
    for (int it = 0; it < a.iterations; ++it) {
        kmeans_assign_kernel<<<g, UB, 0, st>>>(a.X, a.N, a.C, a.n, nullptr, sums, counts);
        kmeans_update_kernel<<<1, 3 * CS_MAX_CLASSES, 0, st>>>(a.C, sums, counts, a.n);
    }
    if (a.assign)
        kmeans_assign_kernel<<<g, UB, 0, st>>>(a.X, a.N, a.C, a.n, a.assign, nullptr, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_kmedians(const KmediansArgs& a, cudaStream_t st) {
    int32_t* members = reinterpret_cast<int32_t*>(a.scratch);
    int32_t* off = members + a.N;
    unsigned* counts = reinterpret_cast<unsigned*>(off + a.n + 1);
    unsigned* cursor = counts + a.n;
    const size_t smem = sizeof(float) * (size_t)a.n * a.k;
    cudaError_t e = set_smem((const void*)kmedians_assign_kernel, smem);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(counts, 0, 2 * sizeof(unsigned) * a.n, st)) != cudaSuccess) return e;
    kmedians_init_kernel<<<(a.n * a.k + UB - 1) / UB, UB, 0, st>>>(a.V, a.N, a.k, a.init, a.n,
                                                                   a.C);
    const int g = grid_for(a.N, a.n_sm);
    for (int it = 0; it < a.iterations; ++it) {
        kmedians_assign_kernel<<<g, UB, smem, st>>>(a.V, a.N, a.k, a.C, a.n, a.work_assign,
                                                    counts);
        class_offsets_kernel<<<1, 32, 0, st>>>(counts, a.n, off, cursor);
        class_scatter_kernel<<<g, UB, 0, st>>>(a.work_assign, a.N, off, cursor, members);
        if ((e = launch_group_medians(a.V, a.N, a.k, a.n, off, members, a.C, st)) != cudaSuccess)
            return e;
    }
    if (a.assign)
        kmedians_assign_kernel<<<g, UB, smem, st>>>(a.V, a.N, a.k, a.C, a.n, a.assign, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_unsup_final(const UnsupFinalArgs& a, cudaStream_t st) {
    const size_t smem = sizeof(float) * (size_t)a.nt * a.k;
    cudaError_t e = set_smem((const void*)unsup_final_kernel, smem);
    if (e != cudaSuccess) return e;
    unsup_final_kernel<<<grid_for(a.P, a.n_sm), UB, smem, st>>>(
        a.img, a.P, a.V, a.k, a.Ccol, a.nc, a.Ctex, a.nt, a.inv2s2, a.inv_beta, a.neglog,
        a.cassign, a.tassign);
    return cudaGetLastError();
}
