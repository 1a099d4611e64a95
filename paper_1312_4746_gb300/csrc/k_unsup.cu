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
// median by radix selection, all classes of a code at once on a cluster of
// blocks that split the points. A class without members keeps its centre.
#include <cooperative_groups.h>

#include <cstdint>

#include "internal.h"

namespace {

constexpr int UB = 256;             // threads per block
constexpr int MB = 512;             // threads per block of the median kernel
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
#pragma unroll 4
    for (int j = 0; j < k; ++j) {
        const float v = V[(size_t)j * N + q];
#pragma unroll
        for (int b = 0; b < CS_MAX_CLASSES; ++b)
            if (b < n) d[b] = __fadd_rn(d[b], fabsf(__fsub_rn(C[b * k + j], v)));
    }
}

__global__ void __launch_bounds__(UB) kmedians_assign_kernel(
    const float* __restrict__ V, int N, int k, const float* __restrict__ Cg, int n,
    int32_t* __restrict__ assign) {
    extern __shared__ float C[];  // n x k
    for (int t = threadIdx.x; t < n * k; t += UB) C[t] = Cg[t];
    __syncthreads();
    for (int q = blockIdx.x * UB + threadIdx.x; q < N; q += gridDim.x * UB) {
        float d[CS_MAX_CLASSES];
        l1_all(V, N, k, q, C, n, d);
        int best = 0;
#pragma unroll
        for (int b = 1; b < CS_MAX_CLASSES; ++b)
            if (b < n && d[b] < d[best]) best = b;
        assign[q] = best;
    }
}

// Order-preserving map of a float's bits to an unsigned key, and back.
__device__ __forceinline__ unsigned key_of(float f) {
    const unsigned u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float float_of(unsigned k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// One cluster of MC blocks per code j: the elementwise median of every class
// over the points assigned to it, by radix selection (four 8-bit passes) on
// all classes at once. Each block histograms its slice of the points (row j
// of V and the assignment, coalesced; updates aggregated per (class, digit)
// within a warp); block 0 of the cluster merges the slices' histograms
// through distributed shared memory, chooses each class's digit and the
// other blocks copy its choice. For an even count the upper middle value is
// the lower one when that key occurs at least twice more from its rank on,
// else the least key above it (one more pass, merged the same way). Classes
// without points keep their centre. The cluster barriers are the hardware's.
constexpr int MC = 4;  // blocks per code

struct MedState {
    unsigned pre[CS_MAX_CLASSES], msk[CS_MAX_CLASSES], rank[CS_MAX_CLASSES];
    unsigned cnt[CS_MAX_CLASSES], eq[CS_MAX_CLASSES], need;
};

__global__ void __cluster_dims__(MC, 1, 1) __launch_bounds__(MB)
    class_median_kernel(const float* __restrict__ V, int N, int k,
                        const int32_t* __restrict__ assign, int n, float* __restrict__ C) {
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    __shared__ unsigned hist[CS_MAX_CLASSES][256];
    __shared__ unsigned merged[CS_MAX_CLASSES][256];
    __shared__ unsigned s_min[CS_MAX_CLASSES];
    __shared__ MedState st;
    const int rank = (int)cluster.block_rank();
    const int j = blockIdx.x / MC;
    const unsigned lane = threadIdx.x & 31u;
    const float* v = V + (size_t)j * N;
    const int chunk = (N + MC - 1) / MC;
    const int q0 = min(rank * chunk, N), q1 = min(q0 + chunk, N);
    if (threadIdx.x < CS_MAX_CLASSES) {
        st.pre[threadIdx.x] = st.msk[threadIdx.x] = st.rank[threadIdx.x] = 0u;
        st.cnt[threadIdx.x] = st.eq[threadIdx.x] = 0u;
        s_min[threadIdx.x] = 0xffffffffu;
    }
    if (threadIdx.x == 0) st.need = 0u;
    for (int pass = 0; pass < 4; ++pass) {
        const int shift = 24 - 8 * pass;
        for (int t = threadIdx.x; t < n * 256; t += MB) hist[t >> 8][t & 255] = 0u;
        __syncthreads();
        for (int q = q0 + threadIdx.x; q < q1; q += MB) {
            const int b = assign[q];
            const unsigned key = key_of(v[q]);
            const bool take = (key & st.msk[b]) == st.pre[b];
            const unsigned dig = (key >> shift) & 255u;
            const unsigned grp =
                __match_any_sync(__activemask(), take ? ((unsigned)b << 8 | dig) : 0xffffffffu);
            if (take && (int)lane == __ffs(grp) - 1) atomicAdd(&hist[b][dig], (unsigned)__popc(grp));
        }
        cluster.sync();  // every slice's histogram is complete
        if (rank == 0) {
            for (int t = threadIdx.x; t < n * 256; t += MB) {
                unsigned m = 0;
                for (int r = 0; r < MC; ++r) m += cluster.map_shared_rank(&hist[0][0], r)[t];
                merged[t >> 8][t & 255] = m;
            }
            __syncthreads();
            if (threadIdx.x < n) {
                const int b = threadIdx.x;
                if (pass == 0) {
                    unsigned m = 0;
                    for (int d = 0; d < 256; ++d) m += merged[b][d];
                    st.cnt[b] = m;
                    st.rank[b] = m ? (m - 1) / 2 : 0u;
                }
                if (st.cnt[b]) {
                    const unsigned r = st.rank[b];
                    unsigned acc = 0;
                    int d = 0;
                    for (; d < 255; ++d) {
                        if (acc + merged[b][d] > r) break;
                        acc += merged[b][d];
                    }
                    st.pre[b] |= (unsigned)d << shift;
                    st.msk[b] |= 255u << shift;
                    st.rank[b] = r - acc;
                    if (pass == 3) {
                        st.eq[b] = merged[b][d];
                        if (!(st.cnt[b] & 1u) && st.eq[b] - st.rank[b] < 2u) atomicOr(&st.need, 1u);
                    }
                }
            }
        }
        cluster.sync();  // block 0's choice is made
        if (rank != 0) {
            const MedState* s0 = cluster.map_shared_rank(&st, 0);
            if (threadIdx.x < CS_MAX_CLASSES) {
                const int b = threadIdx.x;
                st.pre[b] = s0->pre[b];
                st.msk[b] = s0->msk[b];
                st.rank[b] = s0->rank[b];
                st.cnt[b] = s0->cnt[b];
                st.eq[b] = s0->eq[b];
            }
            if (threadIdx.x == 0) st.need = s0->need;
        }
        __syncthreads();
    }
    // block 0 reads the other blocks' minima below: all blocks take part in
    // the same cluster barriers whether or not a class needs the pass
    if (st.need) {  // least key above the lower middle value, for the classes that need it
        for (int q = q0 + threadIdx.x; q < q1; q += MB) {
            const int b = assign[q];
            const unsigned key = key_of(v[q]);
            const bool take = !(st.cnt[b] & 1u) && st.eq[b] - st.rank[b] < 2u && key > st.pre[b];
            const unsigned act = __activemask();
            const unsigned grp = __match_any_sync(act, take ? (unsigned)b : 0xffffffffu);
            const unsigned mn = __reduce_min_sync(grp, take ? key : 0xffffffffu);
            if (take && (int)lane == __ffs(grp) - 1) atomicMin(&s_min[b], mn);
        }
    }
    cluster.sync();  // every slice's minima are in place
    if (rank == 0 && threadIdx.x < n && st.cnt[threadIdx.x]) {
        const int b = threadIdx.x;
        const float lo = float_of(st.pre[b]);
        float out = lo;
        if (!(st.cnt[b] & 1u)) {
            float hi = lo;
            if (st.eq[b] - st.rank[b] < 2u) {
                unsigned m = 0xffffffffu;
                for (int r = 0; r < MC; ++r) m = min(m, cluster.map_shared_rank(&s_min[0], r)[b]);
                hi = float_of(m);
            }
            out = __fmul_rn(0.5f, __fadd_rn(lo, hi));
        }
        C[(size_t)b * k + j] = out;
    }
    cluster.sync();  // no block exits while block 0 may still read its shared memory
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
    const size_t smem = sizeof(float) * (size_t)a.n * a.k;
    cudaError_t e = set_smem((const void*)kmedians_assign_kernel, smem);
    if (e != cudaSuccess) return e;
    kmedians_init_kernel<<<(a.n * a.k + UB - 1) / UB, UB, 0, st>>>(a.V, a.N, a.k, a.init, a.n,
                                                                   a.C);
    const int g = grid_for(a.N, a.n_sm);
    for (int it = 0; it < a.iterations; ++it) {
        kmedians_assign_kernel<<<g, UB, smem, st>>>(a.V, a.N, a.k, a.C, a.n, a.work_assign);
        class_median_kernel<<<a.k * MC, MB, 0, st>>>(a.V, a.N, a.k, a.work_assign, a.n, a.C);
    }
    if (a.assign)
        kmedians_assign_kernel<<<g, UB, smem, st>>>(a.V, a.N, a.k, a.C, a.n, a.assign);
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
