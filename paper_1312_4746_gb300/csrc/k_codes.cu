// Patches, analysis codes and co-support bitmasks (Sec. 2, Sec. 3.1, Eq. 1).
//
// codes_f32_kernel: one thread per pixel of a 16 x 16 tile. The gray tile
// (plus the clamp-to-edge halo) and 32-row chunks of the operator sit in
// shared memory. The patch is built and normalised in FP32, the codes are
// FP32 dot products, and each entry carries a rigorous bound E_j on its
// distance from the exact value (derivation below). Entries with
// | |a_j| - tau | <= E_j cannot be decided in FP32; they go to a guard list
// and codes_guard_kernel recomputes them in double precision following the
// canonical operation order (the same one the CPU oracle uses), so the
// bitmask is exact.
//
// Error bound (u = 2^-24, all quantities per pixel, n = p*p):
//   gray  g = (0.299 R + 0.587 G) + 0.114 B in FP32: |dg| <= 4u Gabs,
//         Gabs = 0.299|R| + 0.587|G| + 0.114|B| (constants' rounding included)
//   v_t = w_t g_t:          |dv_t| <= e_t = 5.1u |w_t| Gabs_t
//   mu  = Kahan sum / n:    |dmu|  <= 3.1u sum|v|/n + sum e/n
//   c_t = v_t - mu:         ||dc||_2 <= 2||e||_2 + 3.1u sum|v|/sqrt(n) + u||c||
//   s = c / ||c|| (ss, sqrt, reciprocal, product):
//                           ||ds||_2 <= 2||dc||/||c|| + (n+7)/2 u
//   a_j = sum_t O_jt s_t:   |da_j| <= ||O_j||_2 (||ds|| + n u (1 + ||ds||))
// The bound is multiplied by 1.25 and widened by tau's FP32 rounding. A
// patch with ||c|| <= 4||dc|| (nearly flat) is recomputed whole.
#include <cuda_bf16.h>

#include <cstdint>

#include "internal.h"
#include "tc_ptx.cuh"

namespace {

constexpr int TILE = 16;
constexpr float U32 = 5.9604645e-08f;  // 2^-24

__global__ void rownorm_kernel(const float* __restrict__ omega, int k, int n,
                               float* __restrict__ rownorm, int* __restrict__ guard_count) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j == 0) *guard_count = 0;
    if (j >= k) return;
    float s = 0.f;
    for (int t = 0; t < n; ++t) s = fmaf(omega[(size_t)j * n + t], omega[(size_t)j * n + t], s);
    // sum of n squares and a square root: relative error <= (n/2 + 2) u
    rownorm[j] = sqrtf(s) * (1.f + (0.5f * n + 2.f) * U32);
}

__device__ __forceinline__ void guard_push(int2* guard, int cap, int* count, int pix, int j) {
    int idx = atomicAdd(count, 1);
    if (idx < cap) guard[idx] = make_int2(pix, j);
}

// Thresholds codes j0 .. j0 + 15 of one pixel (from a tensor-memory load):
// entry j (< k) goes to the co-support word when |a_j| <= tau and it is not
// within its error bound E_j = rn_j ebase + slack of tau; entries within
// the bound are marked in gword for the exact recheck. No branch per entry;
// rn is zero-padded beyond k.
__device__ __forceinline__ void threshold16(const uint32_t (&v)[16], int j0, int k, const float* rn,
                                            float ebase, float tau_f, float tau_slack,
                                            uint32_t& word, uint32_t& gword) {
#pragma unroll
    for (int e = 0; e < 16; ++e) {
        const int j = j0 + e;
        const float aa = fabsf(__uint_as_float(v[e]));
        const float E = rn[j] * ebase + tau_slack;
        const bool g = fabsf(aa - tau_f) <= E;
        const uint32_t m = j < k ? 1u << (j & 31) : 0u;
        word |= (!g && aa <= tau_f) ? m : 0u;
        gword |= g ? m : 0u;
    }
}

// the guard entries of one 32-code word
__device__ __forceinline__ void guard_word(int2* guard, int cap, int* count, int pix, int w,
                                           uint32_t gword) {
    for (uint32_t gm = gword; gm; gm &= gm - 1)
        guard_push(guard, cap, count, pix, 32 * w + __ffs(gm) - 1);
}

template <int P>
__global__ void __launch_bounds__(TILE* TILE)
    codes_f32_kernel(const float* __restrict__ img, int H, int W, const float* __restrict__ omega,
                     int k, const float* __restrict__ mask, const float* __restrict__ rownorm,
                     float tau_f, float tau_slack, float* __restrict__ codes,
                     float* __restrict__ lead16, uint32_t* __restrict__ bitmask,
                     int2* __restrict__ guard, int guard_cap, int* __restrict__ guard_count) {
    constexpr int N = P * P;
    constexpr int NP = (N + 3) & ~3;  // operator rows padded to whole float4s
    constexpr int R = (P - 1) / 2;
    constexpr int TW = TILE + P - 1;
    __shared__ float s_gray[TW * TW];
    __shared__ float s_gabs[TW * TW];
    __shared__ __align__(16) float s_om[32 * NP];
    __shared__ float s_w[N];

    const int tid = threadIdx.y * TILE + threadIdx.x;
    const int y0 = blockIdx.y * TILE, x0 = blockIdx.x * TILE;
    for (int i = tid; i < TW * TW; i += TILE * TILE) {
        int ly = i / TW, lx = i % TW;
        int yy = min(max(y0 + ly - R, 0), H - 1);
        int xx = min(max(x0 + lx - R, 0), W - 1);
        const float* px = img + ((size_t)yy * W + xx) * 3;
        float r = px[0], g = px[1], b = px[2];
        s_gray[i] = __fadd_rn(__fadd_rn(__fmul_rn(0.299f, r), __fmul_rn(0.587f, g)),
                              __fmul_rn(0.114f, b));
        s_gabs[i] = (0.299f * fabsf(r) + 0.587f * fabsf(g) + 0.114f * fabsf(b)) * (1.f + 4 * U32);
    }
    for (int i = tid; i < N; i += TILE * TILE) s_w[i] = mask[i];
    __syncthreads();

    const int y = y0 + threadIdx.y, x = x0 + threadIdx.x;
    const bool live = (y < H) && (x < W);
    const int pix = y * W + x;

    float s[NP];
#pragma unroll
    for (int t = N; t < NP; ++t) s[t] = 0.f;
    float sum = 0.f, kc = 0.f, vabs = 0.f, e2 = 0.f;
#pragma unroll
    for (int dy = 0; dy < P; ++dy)
#pragma unroll
        for (int dx = 0; dx < P; ++dx) {
            const int t = dy * P + dx;
            const int li = (threadIdx.y + dy) * TW + threadIdx.x + dx;
            float v = __fmul_rn(s_w[t], s_gray[li]);
            s[t] = v;
            // Kahan summation of v
            float yk = __fsub_rn(v, kc);
            float tk = __fadd_rn(sum, yk);
            kc = __fsub_rn(__fsub_rn(tk, sum), yk);
            sum = tk;
            vabs += fabsf(v);
            float ew = fabsf(s_w[t]) * s_gabs[li];
            e2 = fmaf(ew, ew, e2);
        }
    const float mu = __fdiv_rn(sum, (float)N);
    float ss = 0.f;
#pragma unroll
    for (int t = 0; t < N; ++t) {
        s[t] = __fsub_rn(s[t], mu);
        ss = fmaf(s[t], s[t], ss);
    }
    const float cn = sqrtf(ss);
    const float dc = (2.f * 5.1f * U32) * sqrtf(e2) * 1.0001f +
                     3.1f * U32 * vabs * rsqrtf((float)N) * 1.0001f + U32 * cn;
    bool whole = !(cn > 4.f * dc);  // nearly flat (or flat): recompute every entry in FP64
    const float inv = whole ? 0.f : __frcp_rn(cn);
#pragma unroll
    for (int t = 0; t < N; ++t) s[t] = __fmul_rn(s[t], inv);
    const float ds = whole ? 0.f : (2.f * dc / cn) * 1.0001f + 0.5f * (N + 7) * U32;
    const float ebase = (ds + (N + 1) * U32 * (1.f + ds)) * 1.25f;

    if (live && whole) guard_push(guard, guard_cap, guard_count, pix, -1);

    const int Wk = (k + 31) >> 5;
    for (int w = 0; w < Wk; ++w) {
        const int j0 = w * 32;
        const int rows = min(32, k - j0);
        __syncthreads();
        for (int i = tid; i < 32 * NP; i += TILE * TILE) {
            const int jj = i / NP, t = i % NP;
            s_om[i] = (jj < rows && t < N) ? omega[(size_t)(j0 + jj) * N + t] : 0.f;
        }
        __syncthreads();
        uint32_t word = 0;
        for (int jj = 0; jj < rows; ++jj) {
            const float4* om = reinterpret_cast<const float4*>(s_om + jj * NP);
            // two interleaved partial sums; the bound below holds for any order
            float a0 = 0.f, a1 = 0.f;
#pragma unroll
            for (int t4 = 0; t4 < NP / 4; ++t4) {
                const float4 o = om[t4];
                a0 = fmaf(o.x, s[4 * t4 + 0], a0);
                a1 = fmaf(o.y, s[4 * t4 + 1], a1);
                a0 = fmaf(o.z, s[4 * t4 + 2], a0);
                a1 = fmaf(o.w, s[4 * t4 + 3], a1);
            }
            const float a = a0 + a1;
            const int j = j0 + jj;
            if (!live) continue;
            const float aa = fabsf(a);
            const float E = rownorm[j] * ebase + tau_slack;
            if (!whole) {
                if (fabsf(aa - tau_f) <= E)
                    guard_push(guard, guard_cap, guard_count, pix, j);
                else if (aa <= tau_f)
                    word |= 1u << jj;
            }
            if (codes) codes[(size_t)pix * k + j] = a;
            if (lead16 && j < 16) lead16[(size_t)pix * 16 + j] = a;
        }
        if (live && bitmask) bitmask[(size_t)pix * Wk + w] = word;
    }
    if (live && lead16)
        for (int j = k; j < 16; ++j) lead16[(size_t)pix * 16 + j] = 0.f;
}

// Canonical double-precision recomputation of guarded entries, one warp per
// entry (entries spread round-robin over the blocks, so over the SMs): the
// patch and code follow the exact operation order of the definition (gray,
// mask product, index-order sums, division by the square root), with every
// operation correctly rounded and no contraction, so the result is
// bit-identical to a sequential evaluation. The element-wise steps (pixel
// loads, products, quotients) run across the lanes; only the three
// index-order sums run on lane 0. An entry (pixel, j) decides code j;
// (pixel, -1) every code of a nearly flat patch (one lane per code). Guarded
// bits were left clear by the codes kernel and are set here.
//
// A code entry is first decided from the same element values with warp-tree
// sums, when that value is clear of tau by a bound that covers both it and
// the index-order evaluation: from the values v_t (identical in both), with
// u = 2^-53, A = sum |v_t|, ss = sum c_t^2, every mean, centring, square,
// root, quotient, product and N-term sum is within
//   |a - a_exact| <= |O_j| (e_s + N u (1 + e_s)),
//   e_s = 2 u sqrt(N) A / sqrt(ss) + (N / 2 + 5) u   (bound on |s - s_exact|)
// of the exact value in either summation order, so the two differ by at most
// twice that; the filter asks for four times (an entry closer to tau, or a
// flat patch, takes the index-order path).
__device__ __forceinline__ double canon_v(const float* __restrict__ img, int H, int W,
                                          const float* __restrict__ mask, int p, int y, int x,
                                          int t) {
    const int r = (p - 1) / 2, dy = t / p, dx = t % p;
    const int yy = min(max(y + dy - r, 0), H - 1), xx = min(max(x + dx - r, 0), W - 1);
    const float* px = img + ((size_t)yy * W + xx) * 3;
    const double gr = __dadd_rn(__dadd_rn(__dmul_rn(0.299, (double)px[0]),
                                          __dmul_rn(0.587, (double)px[1])),
                                __dmul_rn(0.114, (double)px[2]));
    return __dmul_rn((double)mask[t], gr);
}

template <int P>
__global__ void __launch_bounds__(128) codes_guard_kernel(
    const float* __restrict__ img, int H, int W, const float* __restrict__ omega, int k,
    const float* __restrict__ mask, double tau, const int2* __restrict__ guard, int guard_cap,
    const int* __restrict__ guard_count, uint32_t* __restrict__ bitmask, int* __restrict__ d_err) {
    constexpr int N = P * P;
    constexpr int NL = (N + 31) / 32;  // elements per lane
    __shared__ double s_buf[4][N];      // per warp: values for the lane-0 sums
    int cnt = *guard_count;
    if (cnt > guard_cap) {
        if (blockIdx.x == 0 && threadIdx.x == 0 && atomicCAS(d_err, 0, CS_DEVERR_GUARD_FULL) == 0)
            d_err[1] = cnt;
        cnt = guard_cap;
    }
    const int Wk = (k + 31) >> 5;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    double* sb = s_buf[wib];
    auto wsum = [](double v) {  // warp-tree sum, the same value on every lane
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = __dadd_rn(v, __shfl_xor_sync(0xffffffffu, v, o));
        return v;
    };
    for (int e = blockIdx.x + gridDim.x * wib; e < cnt; e += gridDim.x * 4) {
        const int2 g = guard[e];
        const int y = g.x / W, x = g.x % W;
        double c[NL];
        double vv[NL];
#pragma unroll
        for (int u = 0; u < NL; ++u) {
            const int t = lane + 32 * u;
            vv[u] = t < N ? canon_v(img, H, W, mask, P, y, x, t) : 0.0;
            if (t < N) sb[t] = vv[u];
        }
        if (g.y >= 0) {
            // tree-sum filter (see above); warp-uniform decision
            double sv = 0.0, av = 0.0;
#pragma unroll
            for (int u = 0; u < NL; ++u) {
                sv = __dadd_rn(sv, vv[u]);
                av = __dadd_rn(av, fabs(vv[u]));
            }
            const double mu_f = __ddiv_rn(wsum(sv), (double)N), A = wsum(av);
            double sc = 0.0;
#pragma unroll
            for (int u = 0; u < NL; ++u) {
                const int t = lane + 32 * u;
                c[u] = t < N ? __dadd_rn(vv[u], -mu_f) : 0.0;
                sc = __dadd_rn(sc, __dmul_rn(c[u], c[u]));
            }
            const double ss_f = wsum(sc);
            if (ss_f > 0.0) {
                const double nrm_f = __dsqrt_rn(ss_f);
                const float* oj = omega + (size_t)g.y * N;
                double sa = 0.0, so = 0.0;
#pragma unroll
                for (int u = 0; u < NL; ++u) {
                    const int t = lane + 32 * u;
                    const double o = t < N ? (double)oj[t] : 0.0;
                    sa = __dadd_rn(sa, __dmul_rn(o, __ddiv_rn(c[u], nrm_f)));
                    so = __dadd_rn(so, __dmul_rn(o, o));
                }
                const double a_f = wsum(sa), on = __dsqrt_rn(wsum(so));
                const double uu = 1.1102230246251565e-16;  // 2^-53
                const double es = 2.0 * uu * sqrt((double)N) * A / nrm_f + (0.5 * N + 5.0) * uu;
                const double eps = 4.0 * on * (es + N * uu * (1.0 + es)) * 1.01;
                const double aa = fabs(a_f);
                if (aa <= tau - eps || aa > tau + eps) {
                    if (lane == 0 && aa <= tau - eps)
                        atomicOr(bitmask + (size_t)g.x * Wk + (g.y >> 5), 1u << (g.y & 31));
                    __syncwarp();
                    continue;
                }
            }
        }
        __syncwarp();
        double mu = 0.0;
        if (lane == 0) {
            for (int t = 0; t < N; ++t) mu = __dadd_rn(mu, sb[t]);
            mu = __ddiv_rn(mu, (double)N);
        }
        mu = __shfl_sync(0xffffffffu, mu, 0);
#pragma unroll
        for (int u = 0; u < NL; ++u) {
            const int t = lane + 32 * u;
            c[u] = t < N ? __dadd_rn(sb[t], -mu) : 0.0;
        }
        __syncwarp();
#pragma unroll
        for (int u = 0; u < NL; ++u) {
            const int t = lane + 32 * u;
            if (t < N) sb[t] = __dmul_rn(c[u], c[u]);
        }
        __syncwarp();
        double ss = 0.0;
        if (lane == 0)
            for (int t = 0; t < N; ++t) ss = __dadd_rn(ss, sb[t]);
        ss = __shfl_sync(0xffffffffu, ss, 0);
        if (ss == 0.0) {
#pragma unroll
            for (int u = 0; u < NL; ++u) c[u] = 0.0;
        } else {
            const double nrm = __dsqrt_rn(ss);
#pragma unroll
            for (int u = 0; u < NL; ++u) c[u] = __ddiv_rn(c[u], nrm);  // s_t
        }
        __syncwarp();
        if (g.y >= 0) {
            // one code: products across the lanes, the index-order sum on lane 0
            const float* oj = omega + (size_t)g.y * N;
#pragma unroll
            for (int u = 0; u < NL; ++u) {
                const int t = lane + 32 * u;
                if (t < N) sb[t] = __dmul_rn((double)oj[t], c[u]);
            }
            __syncwarp();
            if (lane == 0) {
                double a = 0.0;
                for (int t = 0; t < N; ++t) a = __dadd_rn(a, sb[t]);
                if (fabs(a) <= tau)
                    atomicOr(bitmask + (size_t)g.x * Wk + (g.y >> 5), 1u << (g.y & 31));
            }
        } else {
            // nearly flat patch: every code, one lane per code
#pragma unroll
            for (int u = 0; u < NL; ++u) {
                const int t = lane + 32 * u;
                if (t < N) sb[t] = c[u];
            }
            __syncwarp();
            // up to CG codes per lane at once: independent index-order sums,
            // interleaved so that their latencies overlap
            constexpr int CG = 8;
            for (int j0 = lane; j0 < k; j0 += 32 * CG) {
                double acc[CG];
#pragma unroll
                for (int q = 0; q < CG; ++q) acc[q] = 0.0;
                for (int t = 0; t < N; ++t) {
                    const double st = sb[t];
#pragma unroll
                    for (int q = 0; q < CG; ++q) {
                        const int j = j0 + 32 * q;
                        if (j < k) acc[q] = __dadd_rn(acc[q], __dmul_rn((double)omega[(size_t)j * N + t], st));
                    }
                }
#pragma unroll
                for (int q = 0; q < CG; ++q) {
                    const int j = j0 + 32 * q;
                    if (j < k && fabs(acc[q]) <= tau)
                        atomicOr(bitmask + (size_t)g.x * Wk + (j >> 5), 1u << (j & 31));
                }
            }
        }
        __syncwarp();
    }
}

// Patch order 1 (centre the gray values, mask, centre again, normalise):
// every code of every pixel in double precision, in the canonical index
// order of the reference, one warp per pixel; the co-support test on the
// double value is therefore the reference's decision. Codes and lead16 are
// the double values rounded to FP32.
template <int P>
__global__ void __launch_bounds__(128) codes_fp64_kernel(
    const float* __restrict__ img, int H, int W, const float* __restrict__ omega, int k,
    const float* __restrict__ mask, double tau, float* __restrict__ codes,
    float* __restrict__ lead16, uint32_t* __restrict__ bitmask) {
    constexpr int N = P * P;
    constexpr int NL = (N + 31) / 32;
    constexpr int CG = 4;  // codes per lane in flight
    constexpr int R = (P - 1) / 2;
    __shared__ double s_buf[4][N];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int Wk = (k + 31) >> 5;
    double* sb = s_buf[wib];
    const long long PT = (long long)H * W;
    for (long long q = (long long)blockIdx.x * 4 + wib; q < PT; q += (long long)gridDim.x * 4) {
        const int y = (int)(q / W), x = (int)(q % W);
#pragma unroll
        for (int u = 0; u < NL; ++u) {
            const int t = lane + 32 * u;
            if (t < N) {
                const int yy = min(max(y + t / P - R, 0), H - 1);
                const int xx = min(max(x + t % P - R, 0), W - 1);
                const float* px = img + ((size_t)yy * W + xx) * 3;
                sb[t] = __dadd_rn(__dadd_rn(__dmul_rn(0.299, (double)px[0]),
                                            __dmul_rn(0.587, (double)px[1])),
                                  __dmul_rn(0.114, (double)px[2]));
            }
        }
        __syncwarp();
        double mg = 0.0;
        if (lane == 0) {
            for (int t = 0; t < N; ++t) mg = __dadd_rn(mg, sb[t]);
            mg = __ddiv_rn(mg, (double)N);
        }
        mg = __shfl_sync(0xffffffffu, mg, 0);
        double c[NL];
#pragma unroll
        for (int u = 0; u < NL; ++u) {
            const int t = lane + 32 * u;
            c[u] = t < N ? __dmul_rn((double)mask[t], __dadd_rn(sb[t], -mg)) : 0.0;
        }
        __syncwarp();
#pragma unroll
        for (int u = 0; u < NL; ++u) {
            const int t = lane + 32 * u;
            if (t < N) sb[t] = c[u];
        }
        __syncwarp();
        double mu = 0.0;
        if (lane == 0) {
            for (int t = 0; t < N; ++t) mu = __dadd_rn(mu, sb[t]);
            mu = __ddiv_rn(mu, (double)N);
        }
        mu = __shfl_sync(0xffffffffu, mu, 0);
#pragma unroll
        for (int u = 0; u < NL; ++u) c[u] = __dadd_rn(c[u], -mu);
        __syncwarp();
#pragma unroll
        for (int u = 0; u < NL; ++u) {
            const int t = lane + 32 * u;
            if (t < N) sb[t] = __dmul_rn(c[u], c[u]);
        }
        __syncwarp();
        double ss = 0.0;
        if (lane == 0)
            for (int t = 0; t < N; ++t) ss = __dadd_rn(ss, sb[t]);
        ss = __shfl_sync(0xffffffffu, ss, 0);
        const double nrm = ss == 0.0 ? 0.0 : __dsqrt_rn(ss);
        __syncwarp();
#pragma unroll
        for (int u = 0; u < NL; ++u) {
            const int t = lane + 32 * u;
            if (t < N) sb[t] = ss == 0.0 ? 0.0 : __ddiv_rn(c[u], nrm);  // s_t
        }
        __syncwarp();
        // codes j = jb + 32 g + lane, index-order sums; one ballot per word
        for (int jb = 0; jb < k; jb += 32 * CG) {
            double acc[CG];
#pragma unroll
            for (int g = 0; g < CG; ++g) acc[g] = 0.0;
            for (int t = 0; t < N; ++t) {
                const double st = sb[t];
#pragma unroll
                for (int g = 0; g < CG; ++g) {
                    const int j = jb + 32 * g + lane;
                    if (j < k) acc[g] = __dadd_rn(acc[g], __dmul_rn((double)omega[(size_t)j * N + t], st));
                }
            }
#pragma unroll
            for (int g = 0; g < CG; ++g) {
                const int j = jb + 32 * g + lane;
                const bool in = j < k;
                if (in && codes) codes[q * k + j] = (float)acc[g];
                if (lead16 && j < 16) lead16[q * 16 + j] = in ? (float)acc[g] : 0.f;
                const unsigned word = __ballot_sync(0xffffffffu, in && fabs(acc[g]) <= tau);
                const int w = (jb >> 5) + g;
                if (bitmask && lane == 0 && w < Wk) bitmask[q * Wk + w] = word;
            }
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------- tensor-core codes
//
// codes_tc_kernel: the operator product as a tcgen05 GEMM. One CTA per
// 16 x 8 pixel tile (one thread and one TMEM lane per pixel). The patch is
// built and normalised in FP32 exactly as in codes_f32_kernel (same bound on
// ||ds||) and split into three bf16 pieces, s = s1 + s2 + s3 + r with
// |s2| <= 2^-8 |s|, |s3| <= 2^-16 |s|, |r| <= 2^-24 |s| (each piece the
// bf16 rounding of the exact FP32 remainder); the operator is split the same
// way (O1 + O2 + O3 + q) by omega_split_kernel into the B-operand layout and
// arrives by one bulk (TMA) copy. Six MMA groups accumulate, smallest first,
// O3 s1 + O2 s2 + O1 s3, then O2 s1 + O1 s2, then O1 s1 into FP32 tensor
// memory. Omitted products and residuals contribute at most
// 4.1 * 2^-24 sum_t |O_jt| |s_t|; for the accumulation, each MMA instruction
// is taken to add a relative error of at most 2^-21 of the magnitudes summed
// so far (a margin of 8 over one round-to-nearest; the bf16 x bf16 products
// themselves are exact in FP32), so the KS instructions of the last group
// dominate: KS 2^-21 (1 + 2^-6) plus 5 KS 2^-21 2^-7 for the earlier ones.
// With sum_t |O_jt| |s_t| <= ||O_j|| ||s|| and ||s|| <= 1 + ||ds||, entries
// closer to tau than the bound go to the same guard list and canonical FP64
// recompute as the FP32 form.
constexpr int CT_W = 16, CT_H = 8;  // pixel tile: 128 pixels
constexpr uint64_t CT_WAIT_NS = 1000000000ull;

__host__ __device__ constexpr int ct_ks(int p) { return (p * p + 15) / 16; }
__host__ __device__ constexpr int ct_np(int k) { return (k + 15) / 16 * 16; }
__host__ __device__ constexpr uint32_t ct_cols(int np) {
    return np <= 32 ? 32u : np <= 64 ? 64u : np <= 128 ? 128u : 256u;
}

// Operator pieces in the B-operand layout: 3 KS slabs of np rows x 16 bf16
// (slab piece * KS + s holds piece `piece` of columns 16 s .. 16 s + 15).
__global__ void omega_split_kernel(const float* __restrict__ omega, int k, int n, int ks, int np,
                                   uint8_t* __restrict__ blob, float* __restrict__ rownorm,
                                   int* __restrict__ guard_count) {
    const int total = 3 * ks * np * 16;
    // the first k threads also give the row norms (as rownorm_kernel)
    const int jr = blockIdx.x * blockDim.x + threadIdx.x;
    if (jr == 0) *guard_count = 0;
    if (jr < k) {
        float sq = 0.f;
        for (int t = 0; t < n; ++t) sq = fmaf(omega[(size_t)jr * n + t], omega[(size_t)jr * n + t], sq);
        rownorm[jr] = sqrtf(sq) * (1.f + (0.5f * n + 2.f) * U32);
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const int e = i % 16, j = (i / 16) % np, sl = i / (16 * np);
        const int piece = sl / ks, t = 16 * (sl % ks) + e;
        float rem = (j < k && t < n) ? omega[(size_t)j * n + t] : 0.f;
        uint16_t v = 0;
        for (int q = 0; q <= piece; ++q) {
            const __nv_bfloat16 b = __float2bfloat16_rn(rem);
            v = __bfloat16_as_ushort(b);
            rem -= __bfloat162float(b);  // exact in FP32
        }
        *reinterpret_cast<uint16_t*>(blob + (size_t)sl * np * 32 + tc::slab_off(j, 2 * e)) = v;
    }
}

__device__ __forceinline__ void ct_set_error(int* d_err, int site) {
    if (atomicCAS(d_err, 0, CS_DEVERR_TIMEOUT) == 0) d_err[1] = site;
}

template <int P>
__global__ void __launch_bounds__(128, 4) codes_tc_kernel(
    const float* __restrict__ img, int H, int W, const uint8_t* __restrict__ blob, int k, int np,
    const float* __restrict__ mask, const float* __restrict__ rownorm, float tau_f,
    float tau_slack, float* __restrict__ codes, float* __restrict__ lead16,
    uint32_t* __restrict__ bitmask, int2* __restrict__ guard, int guard_cap,
    int* __restrict__ guard_count, int* __restrict__ d_err) {
    constexpr int N = P * P, R = (P - 1) / 2, KS = ct_ks(P);
    constexpr int GW = CT_W + P - 1, GH = CT_H + P - 1;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t* sa = smem;                                  // A: 3 KS slabs x 4096 B
    uint8_t* sb = smem + 3 * KS * 4096;                  // B: 3 KS slabs x np x 32 B
    uint8_t* misc = sb + 3 * KS * np * 32;               // 32-byte aligned
    uint64_t* bars = reinterpret_cast<uint64_t*>(misc);  // [0] B copy, [1] MMA
    uint32_t* s_tmem = reinterpret_cast<uint32_t*>(misc + 16);
    int* s_flag = reinterpret_cast<int*>(misc + 20);
    float* s_gray = reinterpret_cast<float*>(misc + 32);
    float* s_gabs = s_gray + GW * GH;
    float* s_w = s_gabs + GW * GH;
    float* s_rn = s_w + N;                               // row norms, np

    const int tid = threadIdx.x, warp = tid >> 5;
    const uint32_t ncols = ct_cols(np);
    const uint32_t b_bytes = (uint32_t)(3 * KS * np * 32);
    if (tid == 0) {
        tc::mbar_init(bars + 0, 1);
        tc::mbar_init(bars + 1, 1);
        tc::fence_mbar_init();
        tc::mbar_arrive_expect_tx(bars + 0, b_bytes);
        tc::bulk_g2s(sb, blob, b_bytes, bars + 0);
    }
    if (warp == 0) {
        tc::tmem_alloc(s_tmem, ncols);
        tc::tmem_relinquish();
    }
    const int x0 = blockIdx.x * CT_W, y0 = blockIdx.y * CT_H;
    for (int i = tid; i < GW * GH; i += 128) {
        const int ly = i / GW, lx = i % GW;
        const int yy = min(max(y0 + ly - R, 0), H - 1), xx = min(max(x0 + lx - R, 0), W - 1);
        const float* px = img + ((size_t)yy * W + xx) * 3;
        const float r = px[0], g = px[1], b = px[2];
        s_gray[i] = __fadd_rn(__fadd_rn(__fmul_rn(0.299f, r), __fmul_rn(0.587f, g)),
                              __fmul_rn(0.114f, b));
        s_gabs[i] = (0.299f * fabsf(r) + 0.587f * fabsf(g) + 0.114f * fabsf(b)) * (1.f + 4 * U32);
    }
    for (int i = tid; i < N; i += 128) s_w[i] = mask[i];
    for (int i = tid; i < np; i += 128) s_rn[i] = i < k ? rownorm[i] : 0.f;
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *s_tmem;

    // ---- patch, bound and A operand (row tid) -------------------------------
    const int tx = tid % CT_W, ty = tid / CT_W;
    const int x = x0 + tx, y = y0 + ty;
    const bool live = x < W && y < H;
    const int pix = live ? y * W + x : 0;
    float sum = 0.f, kc = 0.f, vabs = 0.f, e2 = 0.f;
#pragma unroll
    for (int dy = 0; dy < P; ++dy)
#pragma unroll
        for (int dx = 0; dx < P; ++dx) {
            const int t = dy * P + dx, li = (ty + dy) * GW + tx + dx;
            const float v = __fmul_rn(s_w[t], s_gray[li]);
            const float yk = __fsub_rn(v, kc);
            const float tk = __fadd_rn(sum, yk);
            kc = __fsub_rn(__fsub_rn(tk, sum), yk);
            sum = tk;
            vabs += fabsf(v);
            const float ew = fabsf(s_w[t]) * s_gabs[li];
            e2 = fmaf(ew, ew, e2);
        }
    const float mu = __fdiv_rn(sum, (float)N);
    float ss = 0.f;
#pragma unroll
    for (int dy = 0; dy < P; ++dy)
#pragma unroll
        for (int dx = 0; dx < P; ++dx) {
            const int t = dy * P + dx, li = (ty + dy) * GW + tx + dx;
            const float c = __fsub_rn(__fmul_rn(s_w[t], s_gray[li]), mu);
            ss = fmaf(c, c, ss);
        }
    const float cn = sqrtf(ss);
    const float dc = (2.f * 5.1f * U32) * sqrtf(e2) * 1.0001f +
                     3.1f * U32 * vabs * rsqrtf((float)N) * 1.0001f + U32 * cn;
    const bool whole = !(cn > 4.f * dc);
    const float inv = whole ? 0.f : __frcp_rn(cn);
    const float ds = whole ? 0.f : (2.f * dc / cn) * 1.0001f + 0.5f * (N + 7) * U32;
    constexpr float EPS_TC = 4.1f * 5.9604645e-08f + KS * 4.76837158203125e-07f * 1.016f +
                             5 * KS * 4.76837158203125e-07f * 0.0079f;
    const float ebase = (ds + EPS_TC * (1.f + ds)) * 1.25f;
#pragma unroll
    for (int sl = 0; sl < KS; ++sl) {
        uint32_t w1[8], w2[8], w3[8];
#pragma unroll
        for (int e2i = 0; e2i < 8; ++e2i) {
            uint32_t p1 = 0, p2 = 0, p3 = 0;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int t = 16 * sl + 2 * e2i + h;
                float v = 0.f;
                if (t < N && live) {
                    const int li = (ty + t / P) * GW + tx + t % P;
                    v = __fmul_rn(__fsub_rn(__fmul_rn(s_w[t], s_gray[li]), mu), inv);
                }
                const __nv_bfloat16 b1 = __float2bfloat16_rn(v);
                const float r1 = v - __bfloat162float(b1);
                const __nv_bfloat16 b2 = __float2bfloat16_rn(r1);
                const float r2 = r1 - __bfloat162float(b2);
                const __nv_bfloat16 b3 = __float2bfloat16_rn(r2);
                p1 |= (uint32_t)__bfloat16_as_ushort(b1) << (16 * h);
                p2 |= (uint32_t)__bfloat16_as_ushort(b2) << (16 * h);
                p3 |= (uint32_t)__bfloat16_as_ushort(b3) << (16 * h);
            }
            w1[e2i] = p1;
            w2[e2i] = p2;
            w3[e2i] = p3;
        }
        uint8_t* a1 = sa + sl * 4096;
        uint8_t* a2 = sa + (KS + sl) * 4096;
        uint8_t* a3 = sa + (2 * KS + sl) * 4096;
        *reinterpret_cast<uint4*>(a1 + tc::slab_off(tid, 0)) = make_uint4(w1[0], w1[1], w1[2], w1[3]);
        *reinterpret_cast<uint4*>(a1 + tc::slab_off(tid, 16)) = make_uint4(w1[4], w1[5], w1[6], w1[7]);
        *reinterpret_cast<uint4*>(a2 + tc::slab_off(tid, 0)) = make_uint4(w2[0], w2[1], w2[2], w2[3]);
        *reinterpret_cast<uint4*>(a2 + tc::slab_off(tid, 16)) = make_uint4(w2[4], w2[5], w2[6], w2[7]);
        *reinterpret_cast<uint4*>(a3 + tc::slab_off(tid, 0)) = make_uint4(w3[0], w3[1], w3[2], w3[3]);
        *reinterpret_cast<uint4*>(a3 + tc::slab_off(tid, 16)) = make_uint4(w3[4], w3[5], w3[6], w3[7]);
    }
    tc::fence_proxy_async_smem();
    __syncthreads();

    // ---- MMA (one thread) ---------------------------------------------------
    if (tid == 0) {
        int flag = 0;
        if (tc::mbar_wait(bars + 0, 0, tc::globaltimer() + CT_WAIT_NS)) {
            tc::fence_after_sync();
            const uint32_t id = tc::idesc(128, np, 1, 1);
            // (operator piece, patch piece), smallest products first
            const int order[6][2] = {{2, 0}, {1, 1}, {0, 2}, {1, 0}, {0, 1}, {0, 0}};
#pragma unroll
            for (int gi = 0; gi < 6; ++gi)
#pragma unroll
                for (int sl = 0; sl < KS; ++sl)
                    tc::mma_bf16(tmem, tc::smem_desc(sa + (order[gi][1] * KS + sl) * 4096),
                                 tc::smem_desc(sb + (order[gi][0] * KS + sl) * np * 32), id,
                                 gi > 0 || sl > 0);
            tc::mma_commit(bars + 1);
            flag = 1;
        } else {
            ct_set_error(d_err, 21);
            // the copy must land before the CTA may exit
            tc::mbar_wait(bars + 0, 0, tc::globaltimer() + CT_WAIT_NS);
        }
        *s_flag = flag;
    }
    __syncthreads();
    bool ok = *s_flag != 0;
    if (ok && !tc::mbar_wait(bars + 1, 0, tc::globaltimer() + CT_WAIT_NS)) {
        ok = false;
        ct_set_error(d_err, 22);
    }
    ok = __all_sync(0xffffffffu, ok);
    tc::fence_after_sync();

    // ---- epilogue: thresholds, guard list, outputs -------------------------
    if (ok) {
        const int Wk = (k + 31) >> 5;
        const uint32_t lrow = tmem + ((uint32_t)(32 * warp) << 16);
        uint32_t word = 0, gword = 0;
        for (int c = 0; c < np / 16; ++c) {
            uint32_t v[16];
            tc::tmem_ld16(lrow + 16u * c, v);
            tc::tmem_ld_wait();
            threshold16(v, 16 * c, k, s_rn, ebase, tau_f, tau_slack, word, gword);
            if (live && (codes || lead16)) {
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    const int j = 16 * c + e;
                    if (j < k && codes) codes[(size_t)pix * k + j] = __uint_as_float(v[e]);
                    if (j < 16 && j < k && lead16) lead16[(size_t)pix * 16 + j] = __uint_as_float(v[e]);
                }
            }
            if ((c & 1) || c == np / 16 - 1) {
                if (live && !whole) guard_word(guard, guard_cap, guard_count, pix, c >> 1, gword);
                if (live && bitmask) bitmask[(size_t)pix * Wk + (c >> 1)] = whole ? 0u : word;
                word = gword = 0;
            }
        }
        if (live && whole) guard_push(guard, guard_cap, guard_count, pix, -1);
        if (live && lead16)
            for (int j = k; j < 16; ++j) lead16[(size_t)pix * 16 + j] = 0.f;
    } else if (tid == 0 && *s_flag) {
        // MMAs still in flight: they must finish before the tensor memory is freed
        tc::mbar_wait(bars + 1, 0, tc::globaltimer() + CT_WAIT_NS);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, ncols);
    }
}

// codes_tcp_kernel: the same product, persistent (one or two CTAs per SM)
// and pipelined over the 16 x 8 pixel tiles. The operator pieces are copied
// once per CTA. Four builder warps form the normalised patches of tile t + 1
// (each warp two pixel rows, from its own gray window) while the MMAs of
// tile t run, then write its A operand once those MMAs have read the
// previous one; four epilogue warps threshold tile t - 1 from the other of
// two TMEM accumulators; one thread issues the MMAs. The arithmetic per
// pixel and entry is that of codes_tc_kernel.
constexpr int CP_THREADS = 9 * 32;

struct CpOff {
    int b, win, w, rn, prm, bars, misc, total;
};
template <int P>
__host__ __device__ constexpr CpOff cp_off(int np) {
    constexpr int KS = ct_ks(P), N = P * P, WW = CT_W + P - 1, WH = P + 1;
    CpOff o{};
    o.b = 3 * KS * 4096;                                   // A: 3 KS slabs of 128 rows
    o.win = o.b + 3 * KS * np * 32;                        // B: operator pieces
    o.w = o.win + 4 * 2 * WH * WW * 4;                     // builder windows: gray, |gray|
    o.rn = o.w + ((N + 3) & ~3) * 4;                       // patch mask
    o.prm = (o.rn + np * 4 + 15) & ~15;                    // row norms
    o.bars = o.prm + 2 * 128 * 16;                         // per-pixel parameters [2][128]
    o.misc = o.bars + 16 * 8;                              // mbarriers
    o.total = o.misc + 16;                                 // TMEM base, abort flag
    return o;
}

// Bounded wait shared by the roles: gives up after CT_WAIT_NS or once
// another role has aborted.
__device__ __forceinline__ bool cp_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                        int* d_err, int site) {
    const uint64_t deadline = tc::globaltimer() + CT_WAIT_NS;
    for (uint32_t n = 0;; ++n) {
        if (tc::mbar_try_wait(bar, parity, 1000u)) return true;
        if ((n & 63u) == 63u && (*abort_flag || tc::globaltimer() > deadline)) break;
    }
    *abort_flag = 1;
    ct_set_error(d_err, site);
    return false;
}

template <int P>
__global__ void __launch_bounds__(CP_THREADS, P <= 7 ? 2 : 1) codes_tcp_kernel(
    const float* __restrict__ img, int H, int W, const uint8_t* __restrict__ blob, int k, int np,
    const float* __restrict__ mask, const float* __restrict__ rownorm, float tau_f,
    float tau_slack, float* __restrict__ codes, float* __restrict__ lead16,
    uint32_t* __restrict__ bitmask, int2* __restrict__ guard, int guard_cap,
    int* __restrict__ guard_count, int* __restrict__ d_err) {
    constexpr int N = P * P, R = (P - 1) / 2, KS = ct_ks(P);
    constexpr int WW = CT_W + P - 1, WH = P + 1;
    extern __shared__ __align__(1024) uint8_t smem[];
    const CpOff o = cp_off<P>(np);
    uint8_t* sa = smem;
    uint8_t* sb = smem + o.b;
    float* win = reinterpret_cast<float*>(smem + o.win);
    float* s_w = reinterpret_cast<float*>(smem + o.w);
    float* s_rn = reinterpret_cast<float*>(smem + o.rn);
    int4* prm = reinterpret_cast<int4*>(smem + o.prm);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + o.bars);
    uint64_t* b_full = bars + 0;   // operator copy
    uint64_t* a_full = bars + 1;   // builders -> MMA (4 warps)
    uint64_t* a_empty = bars + 2;  // MMA commit -> builders
    uint64_t* t_full = bars + 3;   // [2] MMA commit -> epilogue
    uint64_t* t_empty = bars + 5;  // [2] epilogue (4 warps) -> MMA
    uint64_t* p_full = bars + 7;   // [2] builders (4 warps) -> epilogue: pixel parameters
    uint64_t* p_empty = bars + 9;  // [2] epilogue (4 warps) -> builders
    uint32_t* s_tmem = reinterpret_cast<uint32_t*>(smem + o.misc);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + o.misc + 4);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t ncols = ct_cols(np);
    const uint32_t b_bytes = (uint32_t)(3 * KS * np * 32);
    const int ntx = (W + CT_W - 1) / CT_W, ntiles = ntx * ((H + CT_H - 1) / CT_H);
    if (tid == 0) {
        tc::mbar_init(b_full, 1);
        tc::mbar_init(a_full, 4);
        tc::mbar_init(a_empty, 1);
        for (int b = 0; b < 2; ++b) {
            tc::mbar_init(t_full + b, 1);
            tc::mbar_init(t_empty + b, 4);
            tc::mbar_init(p_full + b, 4);
            tc::mbar_init(p_empty + b, 4);
        }
        *abort_flag = 0;
        tc::fence_mbar_init();
        tc::mbar_arrive_expect_tx(b_full, b_bytes);
        tc::bulk_g2s(sb, blob, b_bytes, b_full);
    }
    if (warp == 8) {
        tc::tmem_alloc(s_tmem, 2 * ncols);
        tc::tmem_relinquish();
    }
    for (int i = tid; i < N; i += CP_THREADS) s_w[i] = mask[i];
    for (int i = tid; i < np; i += CP_THREADS) s_rn[i] = i < k ? rownorm[i] : 0.f;
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *s_tmem;

    if (warp < 4) {
        // ---------------------------------------------------------- builders
        float* wg = win + warp * 2 * WH * WW;  // gray window of pixel rows 2 warp, 2 warp + 1
        float* wa = wg + WH * WW;              // |gray| bound window
        const int r = 32 * warp + lane, tx = lane % CT_W, tyl = lane / CT_W;
        int kk = 0;
        for (int T = blockIdx.x; T < ntiles; T += gridDim.x, ++kk) {
            const int x0 = (T % ntx) * CT_W, y0 = (T / ntx) * CT_H;
#pragma unroll
            for (int i = lane; i < WH * WW; i += 32) {  // every load in flight at once
                const int ly = i / WW, lx = i % WW;
                const int yy = min(max(y0 + 2 * warp + ly - R, 0), H - 1);
                const int xx = min(max(x0 + lx - R, 0), W - 1);
                const float* px = img + ((size_t)yy * W + xx) * 3;
                const float rr = px[0], gg = px[1], bb = px[2];
                wg[i] = __fadd_rn(__fadd_rn(__fmul_rn(0.299f, rr), __fmul_rn(0.587f, gg)),
                                  __fmul_rn(0.114f, bb));
                wa[i] = (0.299f * fabsf(rr) + 0.587f * fabsf(gg) + 0.114f * fabsf(bb)) * (1.f + 4 * U32);
            }
            __syncwarp();
            const int x = x0 + tx, y = y0 + 2 * warp + tyl;
            const bool live = x < W && y < H;
            const int pix = live ? y * W + x : 0;
            float sum = 0.f, kc = 0.f, vabs = 0.f, e2 = 0.f;
#pragma unroll
            for (int dy = 0; dy < P; ++dy)
#pragma unroll
                for (int dx = 0; dx < P; ++dx) {
                    const int t = dy * P + dx, li = (tyl + dy) * WW + tx + dx;
                    const float v = __fmul_rn(s_w[t], wg[li]);
                    const float yk = __fsub_rn(v, kc);
                    const float tk = __fadd_rn(sum, yk);
                    kc = __fsub_rn(__fsub_rn(tk, sum), yk);
                    sum = tk;
                    vabs += fabsf(v);
                    const float ew = fabsf(s_w[t]) * wa[li];
                    e2 = fmaf(ew, ew, e2);
                }
            const float mu = __fdiv_rn(sum, (float)N);
            float ss = 0.f;
#pragma unroll
            for (int dy = 0; dy < P; ++dy)
#pragma unroll
                for (int dx = 0; dx < P; ++dx) {
                    const int t = dy * P + dx, li = (tyl + dy) * WW + tx + dx;
                    const float c = __fsub_rn(__fmul_rn(s_w[t], wg[li]), mu);
                    ss = fmaf(c, c, ss);
                }
            const float cn = sqrtf(ss);
            const float dc = (2.f * 5.1f * U32) * sqrtf(e2) * 1.0001f +
                             3.1f * U32 * vabs * rsqrtf((float)N) * 1.0001f + U32 * cn;
            const bool whole = !(cn > 4.f * dc);
            const float inv = whole ? 0.f : __frcp_rn(cn);
            const float ds = whole ? 0.f : (2.f * dc / cn) * 1.0001f + 0.5f * (N + 7) * U32;
            constexpr float EPS_TC = 4.1f * 5.9604645e-08f + KS * 4.76837158203125e-07f * 1.016f +
                                     5 * KS * 4.76837158203125e-07f * 0.0079f;
            const float ebase = (ds + EPS_TC * (1.f + ds)) * 1.25f;
            // the A operand is free once the previous tile's MMAs have read it
            if (!cp_wait(a_empty, (uint32_t)((kk & 1) ^ 1), abort_flag, d_err, 23)) break;
#pragma unroll
            for (int sl = 0; sl < KS; ++sl) {
                uint32_t w1[8], w2[8], w3[8];
#pragma unroll
                for (int e2i = 0; e2i < 8; ++e2i) {
                    // two codes' inputs at a time, each split into three bf16
                    // pieces (v = b1 + b2 + b3 to 24 bits) by paired conversions
                    float v[2];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int t = 16 * sl + 2 * e2i + h;
                        v[h] = 0.f;
                        if (t < N && live) {
                            const int li = (tyl + t / P) * WW + tx + t % P;
                            v[h] = __fmul_rn(__fsub_rn(__fmul_rn(s_w[t], wg[li]), mu), inv);
                        }
                    }
                    const __nv_bfloat162 b1 = __floats2bfloat162_rn(v[0], v[1]);
                    const float2 f1 = __bfloat1622float2(b1);
                    const float r0 = v[0] - f1.x, r1 = v[1] - f1.y;
                    const __nv_bfloat162 b2 = __floats2bfloat162_rn(r0, r1);
                    const float2 f2 = __bfloat1622float2(b2);
                    const __nv_bfloat162 b3 = __floats2bfloat162_rn(r0 - f2.x, r1 - f2.y);
                    w1[e2i] = *reinterpret_cast<const uint32_t*>(&b1);
                    w2[e2i] = *reinterpret_cast<const uint32_t*>(&b2);
                    w3[e2i] = *reinterpret_cast<const uint32_t*>(&b3);
                }
                uint8_t* a1 = sa + sl * 4096;
                uint8_t* a2 = sa + (KS + sl) * 4096;
                uint8_t* a3 = sa + (2 * KS + sl) * 4096;
                *reinterpret_cast<uint4*>(a1 + tc::slab_off(r, 0)) = make_uint4(w1[0], w1[1], w1[2], w1[3]);
                *reinterpret_cast<uint4*>(a1 + tc::slab_off(r, 16)) = make_uint4(w1[4], w1[5], w1[6], w1[7]);
                *reinterpret_cast<uint4*>(a2 + tc::slab_off(r, 0)) = make_uint4(w2[0], w2[1], w2[2], w2[3]);
                *reinterpret_cast<uint4*>(a2 + tc::slab_off(r, 16)) = make_uint4(w2[4], w2[5], w2[6], w2[7]);
                *reinterpret_cast<uint4*>(a3 + tc::slab_off(r, 0)) = make_uint4(w3[0], w3[1], w3[2], w3[3]);
                *reinterpret_cast<uint4*>(a3 + tc::slab_off(r, 16)) = make_uint4(w3[4], w3[5], w3[6], w3[7]);
            }
            tc::fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(a_full);
            // this pixel's parameters for the epilogue
            const int pb = kk & 1;
            if (!cp_wait(p_empty + pb, (uint32_t)(((kk >> 1) & 1) ^ 1), abort_flag, d_err, 24)) break;
            prm[pb * 128 + r] = make_int4(live ? pix : -1, whole ? 1 : 0, __float_as_int(ebase), 0);
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(p_full + pb);
        }
    } else if (warp < 8) {
        // ---------------------------------------------------------- epilogue
        const int q = warp & 3;
        const uint32_t lrow = tmem + ((uint32_t)(32 * q) << 16);
        const int Wk = (k + 31) >> 5, nch = np / 16;
        int kk = 0;
        for (int T = blockIdx.x; T < ntiles; T += gridDim.x, ++kk) {
            const int b = kk & 1;
            if (!cp_wait(p_full + b, (uint32_t)((kk >> 1) & 1), abort_flag, d_err, 25)) break;
            const int4 pp = prm[b * 128 + 32 * q + lane];
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(p_empty + b);
            if (!cp_wait(t_full + b, (uint32_t)((kk >> 1) & 1), abort_flag, d_err, 26)) break;
            tc::fence_after_sync();
            const bool live = pp.x >= 0, whole = pp.y != 0;
            const int pix = live ? pp.x : 0;
            const float ebase = __int_as_float(pp.z);
            uint32_t word = 0, gword = 0;
            for (int c = 0; c < nch; ++c) {
                uint32_t v[16];
                tc::tmem_ld16(lrow + (uint32_t)(b * ncols) + 16u * c, v);
                tc::tmem_ld_wait();
                threshold16(v, 16 * c, k, s_rn, ebase, tau_f, tau_slack, word, gword);
                if (live && (codes || lead16)) {
#pragma unroll
                    for (int e = 0; e < 16; ++e) {
                        const int j = 16 * c + e;
                        if (j < k && codes) codes[(size_t)pix * k + j] = __uint_as_float(v[e]);
                        if (j < 16 && j < k && lead16)
                            lead16[(size_t)pix * 16 + j] = __uint_as_float(v[e]);
                    }
                }
                if ((c & 1) || c == nch - 1) {
                    if (live && !whole) guard_word(guard, guard_cap, guard_count, pix, c >> 1, gword);
                    if (live && bitmask) bitmask[(size_t)pix * Wk + (c >> 1)] = whole ? 0u : word;
                    word = gword = 0;
                }
            }
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(t_empty + b);
            if (live && whole) guard_push(guard, guard_cap, guard_count, pix, -1);
            if (live && lead16)
                for (int j = k; j < 16; ++j) lead16[(size_t)pix * 16 + j] = 0.f;
        }
    } else if (lane == 0) {
        // ---------------------------------------------------------- MMA issuer
        long long last = -1;
        if (cp_wait(b_full, 0, abort_flag, d_err, 21)) {
            const uint32_t id = tc::idesc(128, np, 1, 1);
            int kk = 0;
            for (int T = blockIdx.x; T < ntiles; T += gridDim.x, ++kk) {
                const int b = kk & 1;
                if (!cp_wait(a_full, (uint32_t)(kk & 1), abort_flag, d_err, 22) ||
                    !cp_wait(t_empty + b, (uint32_t)(((kk >> 1) & 1) ^ 1), abort_flag, d_err, 27))
                    break;
                tc::fence_after_sync();
                const uint32_t d = tmem + (uint32_t)(b * ncols);
                // (operator piece, patch piece), smallest products first
                const int order[6][2] = {{2, 0}, {1, 1}, {0, 2}, {1, 0}, {0, 1}, {0, 0}};
#pragma unroll
                for (int gi = 0; gi < 6; ++gi)
#pragma unroll
                    for (int sl = 0; sl < KS; ++sl)
                        tc::mma_bf16(d, tc::smem_desc(sa + (order[gi][1] * KS + sl) * 4096),
                                     tc::smem_desc(sb + (order[gi][0] * KS + sl) * np * 32), id,
                                     gi > 0 || sl > 0);
                tc::mma_commit(a_empty);
                tc::mma_commit(t_full + b);
                last = kk;
            }
        } else {
            // the copy must land before the CTA may exit
            tc::mbar_wait(b_full, 0, tc::globaltimer() + CT_WAIT_NS);
        }
        // drain: the last MMAs must finish before the tensor memory is freed
        if (last >= 0)
            tc::mbar_wait(t_full + (int)(last & 1), (uint32_t)((last >> 1) & 1),
                          tc::globaltimer() + CT_WAIT_NS);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 8) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, 2 * ncols);
    }
}

template <int P>
size_t ct_smem(int np) {
    constexpr int N = P * P, KS = ct_ks(P), GW = CT_W + P - 1, GH = CT_H + P - 1;
    size_t b = 3 * KS * 4096 + 3 * KS * (size_t)np * 32 + 32 + 4 * (2 * GW * GH + N + np);
    b = (b + 15) / 16 * 16;
    // at most 512 / ncols CTAs per SM, so that tensor-memory allocations never wait
    const int per_sm = 512 / (int)ct_cols(np);
    if (per_sm < 16) {
        const size_t floor_b = 233472 / (per_sm + 1) - 1024 + 16;
        if (b < floor_b) b = floor_b;
    }
    return b;
}

template <int P>
cudaError_t launch_tc_p(const CodesArgs& a, cudaStream_t st) {
    const int np = ct_np(a.k);
    const size_t smem = ct_smem<P>(np);
    cudaError_t e = cudaFuncSetAttribute(codes_tc_kernel<P>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int total = 3 * ct_ks(P) * np * 16;
    omega_split_kernel<<<(total + 255) / 256, 256, 0, st>>>(a.omega, a.k, P * P, ct_ks(P), np,
                                                           a.omega_blob, a.rownorm, a.guard_count);
    const float tau_f = (float)a.tau;
    const float slack = fabsf(tau_f - (float)a.tau) + 2.f * U32 * tau_f + 1e-12f;
    // persistent and pipelined where its layout fits (at most two CTAs per
    // SM: TMEM holds two accumulators each), else one CTA per pixel tile
    const int ncols2 = 2 * (int)ct_cols(np);
    size_t psmem = (size_t)cp_off<P>(np).total;
    int per_sm = 512 / ncols2;
    const int per_sm_smem = (int)(233472 / (psmem + 1024));
    if (per_sm > per_sm_smem) per_sm = per_sm_smem;
    if (per_sm > (P <= 7 ? 2 : 1)) per_sm = P <= 7 ? 2 : 1;  // registers (launch bounds)
    if (per_sm < 1) {
        dim3 grd((a.W + CT_W - 1) / CT_W, (a.H + CT_H - 1) / CT_H);
        codes_tc_kernel<P><<<grd, 128, smem, st>>>(a.img, a.H, a.W, a.omega_blob, a.k, np, a.mask,
                                                   a.rownorm, tau_f, slack, a.codes, a.lead16,
                                                   a.bitmask, a.guard, a.guard_cap, a.guard_count,
                                                   a.d_err);
        return cudaGetLastError();
    }
    const size_t floor_b = 233472 / (per_sm + 1) - 1024 + 16;  // no further CTA fits
    if (psmem < floor_b) psmem = floor_b;
    e = cudaFuncSetAttribute(codes_tcp_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)psmem);
    if (e != cudaSuccess) return e;
    int dev = 0, n_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return e;
    const int ntiles = ((a.W + CT_W - 1) / CT_W) * ((a.H + CT_H - 1) / CT_H);
    const int grid = ntiles < per_sm * n_sm ? ntiles : per_sm * n_sm;
    codes_tcp_kernel<P><<<grid, CP_THREADS, psmem, st>>>(
        a.img, a.H, a.W, a.omega_blob, a.k, np, a.mask, a.rownorm, tau_f, slack, a.codes,
        a.lead16, a.bitmask, a.guard, a.guard_cap, a.guard_count, a.d_err);
    return cudaGetLastError();
}

__global__ void cosupport_kernel(const float* __restrict__ codes, long long total, int k,
                                 double tau, uint32_t* __restrict__ bitmask) {
    // one thread per output word
    const int Wk = (k + 31) >> 5;
    long long nw = total / k * Wk;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nw;
         i += (long long)gridDim.x * blockDim.x) {
        long long q = i / Wk;
        int w = (int)(i % Wk);
        uint32_t word = 0;
        for (int b = 0; b < 32; ++b) {
            int j = w * 32 + b;
            if (j >= k) break;
            if (fabs((double)codes[q * k + j]) <= tau) word |= 1u << b;
        }
        bitmask[i] = word;
    }
}

template <int P>
cudaError_t launch_p(const CodesArgs& a, cudaStream_t st) {
    dim3 blk(TILE, TILE), grd((a.W + TILE - 1) / TILE, (a.H + TILE - 1) / TILE);
    const float tau_f = (float)a.tau;
    const float slack = fabsf(tau_f - (float)a.tau) + 2.f * U32 * tau_f + 1e-12f;
    codes_f32_kernel<P><<<grd, blk, 0, st>>>(a.img, a.H, a.W, a.omega, a.k, a.mask, a.rownorm,
                                             tau_f, slack, a.codes, a.lead16, a.bitmask, a.guard,
                                             a.guard_cap, a.guard_count);
    return cudaGetLastError();
}

}  // namespace

bool codes_tc_supported(int k, int p) { return k >= 1 && k <= 256 && p >= 3 && p <= 9 && (p & 1); }

size_t codes_tc_blob_bytes(int k, int p) { return (size_t)3 * ct_ks(p) * ct_np(k) * 32; }

cudaError_t launch_codes(const CodesArgs& a, cudaStream_t st) {
    const int n = a.p * a.p;
    if (a.order == 1) {
        const long long PT = (long long)a.H * a.W;
        const int grid = (int)((PT + 3) / 4 < 152 * 16 ? (PT + 3) / 4 : 152 * 16);
        switch (a.p) {
            case 3: codes_fp64_kernel<3><<<grid, 128, 0, st>>>(a.img, a.H, a.W, a.omega, a.k, a.mask, a.tau, a.codes, a.lead16, a.bitmask); break;
            case 5: codes_fp64_kernel<5><<<grid, 128, 0, st>>>(a.img, a.H, a.W, a.omega, a.k, a.mask, a.tau, a.codes, a.lead16, a.bitmask); break;
            case 7: codes_fp64_kernel<7><<<grid, 128, 0, st>>>(a.img, a.H, a.W, a.omega, a.k, a.mask, a.tau, a.codes, a.lead16, a.bitmask); break;
            case 9: codes_fp64_kernel<9><<<grid, 128, 0, st>>>(a.img, a.H, a.W, a.omega, a.k, a.mask, a.tau, a.codes, a.lead16, a.bitmask); break;
            default: return cudaErrorInvalidValue;
        }
        return cudaGetLastError();
    }
    // (the tensor-core form's operator split also gives the row norms)
    if (!a.tc)
        rownorm_kernel<<<(a.k + 127) / 128, 128, 0, st>>>(a.omega, a.k, n, a.rownorm, a.guard_count);
    cudaError_t e;
    if (a.tc) {
        if (!a.omega_blob || !codes_tc_supported(a.k, a.p)) return cudaErrorInvalidValue;
        switch (a.p) {
            case 3: e = launch_tc_p<3>(a, st); break;
            case 5: e = launch_tc_p<5>(a, st); break;
            case 7: e = launch_tc_p<7>(a, st); break;
            case 9: e = launch_tc_p<9>(a, st); break;
            default: return cudaErrorInvalidValue;
        }
    } else {
        switch (a.p) {
            case 3: e = launch_p<3>(a, st); break;
            case 5: e = launch_p<5>(a, st); break;
            case 7: e = launch_p<7>(a, st); break;
            case 9: e = launch_p<9>(a, st); break;
            default: return cudaErrorInvalidValue;
        }
    }
    if (e != cudaSuccess) return e;
    if (!a.bitmask) return cudaSuccess;
#define CS_GUARD(PP)                                                                        \
    case PP:                                                                                \
        codes_guard_kernel<PP><<<152 * 4, 128, 0, st>>>(a.img, a.H, a.W, a.omega, a.k, a.mask, \
                                                        a.tau, a.guard, a.guard_cap,          \
                                                        a.guard_count, a.bitmask, a.d_err);   \
        break;
    switch (a.p) {
        CS_GUARD(3)
        CS_GUARD(5)
        CS_GUARD(7)
        CS_GUARD(9)
        default: return cudaErrorInvalidValue;
    }
#undef CS_GUARD
    return cudaGetLastError();
}

cudaError_t launch_cosupport(const float* codes, long long P, int k, double tau,
                             uint32_t* bitmask, cudaStream_t st) {
    cosupport_kernel<<<152 * 8, 256, 0, st>>>(codes, P * k, k, tau, bitmask);
    return cudaGetLastError();
}
