// Convex multilabel segmentation on the data term (Sec. 4): the relaxed
// energy of Eq. (energy1) / Eq. (sets) minimised by the primal-dual
// iteration of Eq. (algo), then binarised by argmax.
//
// Discretisation (the paper gives none): forward differences with a zero
// difference across the last row / column for grad, its negative adjoint for
// div; edge weight g(x) = exp(-|grad I(x)| / gamma) / (2 gamma) with |grad I|
// the Euclidean norm of the forward differences of the three channels of
// 255 I; step sizes by diagonal preconditioning: 1/2 for xi and mu, 1/5 for
// u, 1/|Omega| for m; start u = 1/n, m = 1, xi = mu = 0.
//
// One persistent cooperative launch runs every iteration. Each block owns a
// contiguous range of pixels (all labels) and keeps its own copy of m in
// shared memory; per iteration: the dual step (xi, mu and the block's sums of
// mu per label), a grid barrier, the m step (every block sums the per-block
// parts in the same fixed order, so all copies agree), the primal step (u by
// Michelot's simplex projection per pixel, over-relaxed copy ub), a grid
// barrier. The working set (about 6 n |Omega| floats) stays in L2. The grid
// barriers are bounded waits: on timeout the kernel records the site in the
// error word, raises an abort flag that every other block sees, and returns.
#include <atomic>
#include <cstdint>
#include <mutex>

#include "internal.h"

namespace {

constexpr int SB = 512;                         // threads per block
constexpr int NW = SB / 32;
constexpr unsigned long long SEG_WAIT_NS = 1000000000ull;  // 1 s per barrier

__device__ __forceinline__ uint64_t seg_clock() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid barrier on a monotonic arrival counter: barrier number `k` (from 1)
// completes when the counter reaches k * gridDim.x. bar[0] = counter,
// bar[1] = abort flag. Returns false (for the whole block) when this block
// gave up or another block raised the abort flag. `arrive` false (the
// timeout-path test) skips this block's arrival, so that no block's wait
// completes: every block gives up after `wait_ns` or on the abort flag.
__device__ bool grid_barrier(unsigned* bar, unsigned k, int* d_err, int site, int* s_ok,
                             uint64_t wait_ns, bool arrive = true) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (arrive) atomicAdd(bar, 1u);
        const unsigned target = k * gridDim.x;
        const uint64_t deadline = seg_clock() + wait_ns;
        int ok = 1;
        for (unsigned n = 0;; ++n) {
            if ((int)(ld_acquire(bar) - target) >= 0) break;
            if ((n & 63u) == 63u) {
                if (ld_acquire(bar + 1)) {
                    ok = 0;
                    break;
                }
                if (seg_clock() > deadline) {
                    if (atomicCAS(d_err, 0, CS_DEVERR_TIMEOUT) == 0) d_err[1] = site;
                    atomicExch(bar + 1, 1u);
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

// State that other blocks write during the launch (u, ub, px, py, mu, parts)
// is read through plain pointers (no read-only cache path).
struct SegState {
    const float* f;
    const float* img;
    float* u;
    float* ub;
    float* px;
    float* py;
    float* mu;
    float* bound;
    float* parts;  // n x gridDim.x sums of mu
    unsigned* bar;
    int32_t* labels;
    int* d_err;
    int H, W, n, iterations;
    float lambda, nu, gamma;
    uint64_t wait_ns;  // limit of each grid-barrier wait
    bool stall;        // the last block skips its arrival at the first barrier of the iterations
};

// N: the label count when it is at most 8 (every label loop unrolled
// exactly), else an upper bound (16 or CS_MAX_LABELS, loops guarded by
// i < n). I: the element index type, int when n |Omega| fits. The dual step
// takes the labels in groups of 4 so that each group's loads are in flight
// together; the primal step holds the pixel's labels in registers.
template <int N, typename I>
__global__ void __launch_bounds__(SB, 2) seg_solve_kernel(SegState S) {
    constexpr bool EXACT = N <= 8;
    __shared__ float red[CS_MAX_LABELS][NW];
    __shared__ float s_m[CS_MAX_LABELS], s_mb[CS_MAX_LABELS];
    __shared__ int s_ok;
    const int P = S.H * S.W;  // H W < 2^31 (checked by the caller)
    const int n = EXACT ? N : S.n;
    const int W = S.W, H = S.H;
    const int G = gridDim.x, b = blockIdx.x;
    const int chunk = (int)(((long long)P + G - 1) / G);
    const int q0 = (int)((long long)b * chunk < P ? (long long)b * chunk : P);
    const int q1 = (int)((long long)q0 + chunk < P ? (long long)q0 + chunk : P);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    // edge weight bound lambda g / 2 and the start point, own pixels
    for (int q = q0 + threadIdx.x; q < q1; q += SB) {
        const int y = q / W, x = q - y * W;
        float s = 0.f;
        for (int c = 0; c < 3; ++c) {
            const float v = 255.f * S.img[(size_t)q * 3 + c];
            const float dx = x + 1 < W ? 255.f * S.img[(size_t)(q + 1) * 3 + c] - v : 0.f;
            const float dy = y + 1 < H ? 255.f * S.img[(size_t)(q + W) * 3 + c] - v : 0.f;
            s = fmaf(dx, dx, fmaf(dy, dy, s));
        }
        S.bound[q] = 0.5f * S.lambda * (expf(-sqrtf(s) / S.gamma) / (2.f * S.gamma));
        for (int i = 0; i < n; ++i) {
            const I e = (I)i * P + q;
            S.u[e] = 1.f / (float)n;
            S.ub[e] = 1.f / (float)n;
            S.px[e] = 0.f;
            S.py[e] = 0.f;
            S.mu[e] = 0.f;
        }
    }
    for (int i = threadIdx.x; i < n; i += SB) s_m[i] = s_mb[i] = 1.f;
    unsigned nbar = 0;
    if (!grid_barrier(S.bar, ++nbar, S.d_err, 40, &s_ok, S.wait_ns)) return;

    const float inv_area = 1.f / (float)P;
    for (int it = 0; it < S.iterations; ++it) {
        // dual step: xi <- Pi_Kg(xi + 1/2 grad ub), mu <- min(0, mu + 1/2 (mb - ub))
#pragma unroll 1
        for (int i0 = 0; i0 < n; i0 += 4) {
            float acc[4] = {0.f, 0.f, 0.f, 0.f};
            for (int q = q0 + threadIdx.x; q < q1; q += SB) {
                const int y = q / W, x = q - y * W;
                const bool hr = x + 1 < W, hd = y + 1 < H;
                const float bd = S.bound[q];
                float c[4], gx[4], gy[4], ax[4], ay[4], m0[4];
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (i0 + j < n) {
                        const I e = (I)(i0 + j) * P + q;
                        c[j] = S.ub[e];
                        gx[j] = hr ? S.ub[e + 1] : 0.f;
                        gy[j] = hd ? S.ub[e + W] : 0.f;
                        ax[j] = S.px[e];
                        ay[j] = S.py[e];
                        m0[j] = S.mu[e];
                    }
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (i0 + j < n) {
                        const I e = (I)(i0 + j) * P + q;
                        float vx = ax[j] + 0.5f * (hr ? gx[j] - c[j] : 0.f);
                        float vy = ay[j] + 0.5f * (hd ? gy[j] - c[j] : 0.f);
                        const float nrm = sqrtf(vx * vx + vy * vy);
                        if (nrm > bd) {
                            const float sc = bd > 0.f ? __fdividef(bd, nrm) : 0.f;
                            vx *= sc;
                            vy *= sc;
                        }
                        S.px[e] = vx;
                        S.py[e] = vy;
                        const float m = fminf(0.f, m0[j] + 0.5f * (s_mb[i0 + j] - c[j]));
                        S.mu[e] = m;
                        acc[j] += m;
                    }
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float a = acc[j];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
                if (lane == 0 && i0 + j < n) red[i0 + j][warp] = a;
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += SB) {
            float s = 0.f;
            for (int w = 0; w < NW; ++w) s += red[i][w];
            S.parts[(size_t)i * G + b] = s;
        }
        if (!grid_barrier(S.bar, ++nbar, S.d_err, 41, &s_ok, S.wait_ns,
                          !(S.stall && it == 0 && b == G - 1)))
            return;

        // m step: m <- clamp(m - (nu + sum mu) / |Omega|, 0, 1), mb = 2 m_new - m;
        // one warp per label, the same summation order in every block
        for (int i = warp; i < n; i += NW) {
            float s = 0.f;
            for (int k = lane; k < G; k += 32) s += S.parts[(size_t)i * G + k];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) {
                const float mo = s_m[i];
                const float mn = fminf(1.f, fmaxf(0.f, mo - inv_area * (S.nu + s)));
                s_mb[i] = 2.f * mn - mo;
                s_m[i] = mn;
            }
        }

        // primal step per pixel: u <- Pi_simplex(u - 1/5 (-div xi + f - mu)) by
        // Michelot's algorithm over the labels, ub = 2 u_new - u
        for (int q = q0 + threadIdx.x; q < q1; q += SB) {
            const int y = q / W, x = q - y * W;
            float v[N], uo[N];
            unsigned long long active = 0;
#pragma unroll
            for (int i = 0; i < N; ++i)
                if (EXACT || i < n) {
                    const I e = (I)i * P + q;
                    const float pxr = x + 1 < W ? S.px[e] : 0.f;
                    const float pxl = x > 0 ? S.px[e - 1] : 0.f;
                    const float pyd = y + 1 < H ? S.py[e] : 0.f;
                    const float pyu = y > 0 ? S.py[e - W] : 0.f;
                    const float d = (pxr - pxl) + (pyd - pyu);  // div xi
                    uo[i] = S.u[e];
                    v[i] = uo[i] - 0.2f * (-d + S.f[e] - S.mu[e]);
                    active |= 1ull << i;
                }
            // Michelot: project onto the active indices' hyperplane, drop negatives
            float shift = 0.f;
            for (int round = 0; round < n; ++round) {
                float s = 0.f;
                int cnt = 0;
#pragma unroll
                for (int i = 0; i < N; ++i)
                    if ((active >> i) & 1ull) {
                        s += v[i];
                        ++cnt;
                    }
                shift = __fdividef(s - 1.f, (float)cnt);
                bool drop = false;
#pragma unroll
                for (int i = 0; i < N; ++i)
                    if (((active >> i) & 1ull) && v[i] - shift < 0.f) {
                        active &= ~(1ull << i);
                        drop = true;
                    }
                if (!drop) break;
            }
#pragma unroll
            for (int i = 0; i < N; ++i)
                if (EXACT || i < n) {
                    const I e = (I)i * P + q;
                    const float un = ((active >> i) & 1ull) ? v[i] - shift : 0.f;
                    S.ub[e] = 2.f * un - uo[i];
                    S.u[e] = un;
                }
        }
        if (!grid_barrier(S.bar, ++nbar, S.d_err, 42, &s_ok, S.wait_ns)) return;
    }

    if (S.labels)
        for (int q = q0 + threadIdx.x; q < q1; q += SB) {
            int best = 0;
            float bv = S.u[q];
            for (int i = 1; i < n; ++i) {
                const float v = S.u[(I)i * P + q];
                if (v > bv) {
                    bv = v;
                    best = i;
                }
            }
            S.labels[q] = best;
        }
}

using SegKernel = void (*)(SegState);

template <typename I>
SegKernel seg_kernel_t(int n) {
    switch (n) {
        case 1: return seg_solve_kernel<1, I>;
        case 2: return seg_solve_kernel<2, I>;
        case 3: return seg_solve_kernel<3, I>;
        case 4: return seg_solve_kernel<4, I>;
        case 5: return seg_solve_kernel<5, I>;
        case 6: return seg_solve_kernel<6, I>;
        case 7: return seg_solve_kernel<7, I>;
        case 8: return seg_solve_kernel<8, I>;
        default: return n <= 16 ? seg_solve_kernel<16, I> : seg_solve_kernel<CS_MAX_LABELS, I>;
    }
}

// the element index n P + P (the last label's plane plus a row) fits an int?
bool seg_narrow(long long P, int n) { return (long long)(n + 1) * P < (1ll << 31); }

SegKernel seg_kernel(long long P, int n) {
    return seg_narrow(P, n) ? seg_kernel_t<int>(n) : seg_kernel_t<long long>(n);
}

int seg_grid(long long P, int n, int n_sm) {
    // co-resident blocks per SM, per variant (labels 1..8, 16, 64; narrow /
    // wide index); -1 until queried (calls from several threads store the
    // same value)
    static std::atomic<int> per_sm[2][10];
    static std::once_flag init;
    std::call_once(init, [] {
        for (auto& row : per_sm)
            for (auto& v : row) v.store(-1);
    });
    const int v = n <= 8 ? n - 1 : n <= 16 ? 8 : 9;
    std::atomic<int>& slot = per_sm[seg_narrow(P, n) ? 0 : 1][v];
    int nb = slot.load();
    if (nb < 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, seg_kernel(P, n), SB, 0) !=
            cudaSuccess)
            nb = 0;
        slot.store(nb);
    }
    const int k = nb < 2 ? nb : 2;
    return k * n_sm;
}

}  // namespace

size_t seg_scratch_bytes(long long P, int n, int nblk) {
    return sizeof(float) * ((size_t)4 * n * P + (size_t)P + (size_t)n * nblk) + 1024;
}

int seg_blocks(long long P, int n, int n_sm) {
    const long long need = (P + SB - 1) / SB;
    const int g = seg_grid(P, n, n_sm);
    return (int)(need < g ? need : g);
}

cudaError_t launch_segment(const SegArgs& a, cudaStream_t st) {
    const long long P = (long long)a.H * a.W;
    const int n = a.n_labels;
    if (a.nblk < 1) return cudaErrorInvalidConfiguration;
    SegState S;
    S.f = a.f;
    S.img = a.img;
    S.u = a.u;
    S.ub = a.scratch;
    S.px = S.ub + (size_t)n * P;
    S.py = S.px + (size_t)n * P;
    S.mu = S.py + (size_t)n * P;
    S.bound = S.mu + (size_t)n * P;
    S.parts = S.bound + P;
    // the barrier words sit 256-byte aligned after the parts
    const uintptr_t end = reinterpret_cast<uintptr_t>(S.parts + (size_t)n * a.nblk);
    S.bar = reinterpret_cast<unsigned*>((end + 255) & ~(uintptr_t)255);
    S.labels = a.labels;
    S.d_err = a.d_err;
    S.H = a.H;
    S.W = a.W;
    S.n = n;
    S.iterations = a.iterations;
    S.lambda = a.lambda;
    S.nu = a.nu;
    S.gamma = a.gamma;
    S.wait_ns = a.wait_ns ? a.wait_ns : SEG_WAIT_NS;
    S.stall = a.stall && a.iterations > 0;
    cudaError_t e = cudaMemsetAsync(S.bar, 0, 2 * sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    void* args[] = {&S};
    return cudaLaunchCooperativeKernel((const void*)seg_kernel(P, n), dim3(a.nblk), dim3(SB), args,
                                       0, st);
}
