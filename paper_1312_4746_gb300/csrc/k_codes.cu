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
#include <cstdint>

#include "internal.h"

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
// entry: the patch and code follow the exact operation order of the
// definition (gray, mask product, index-order sums, division by the square
// root), with every operation correctly rounded and no contraction. The
// element-wise steps run across the lanes; every sum runs on lane 0 in index
// order, so the result is bit-identical to a sequential evaluation.
__global__ void codes_guard_kernel(const float* __restrict__ img, int H, int W,
                                   const float* __restrict__ omega, int k,
                                   const float* __restrict__ mask, int p, double tau,
                                   const int2* __restrict__ guard, int guard_cap,
                                   const int* __restrict__ guard_count,
                                   uint32_t* __restrict__ bitmask, int* __restrict__ d_err) {
    __shared__ double s_s[4][81];
    __shared__ double s_ab[4];
    int cnt = *guard_count;
    if (cnt > guard_cap) {
        if (blockIdx.x == 0 && threadIdx.x == 0 && atomicCAS(d_err, 0, CS_DEVERR_GUARD_FULL) == 0)
            d_err[1] = cnt;
        cnt = guard_cap;
    }
    const int n = p * p, r = (p - 1) / 2, Wk = (k + 31) >> 5;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    double* s = s_s[wib];
    const int warps = gridDim.x * (blockDim.x >> 5);
    for (int e = blockIdx.x * (blockDim.x >> 5) + wib; e < cnt; e += warps) {
        const int2 g = guard[e];
        const int y = g.x / W, x = g.x % W;
        for (int t = lane; t < n; t += 32) {
            const int dy = t / p, dx = t % p;
            const int yy = min(max(y + dy - r, 0), H - 1), xx = min(max(x + dx - r, 0), W - 1);
            const float* px = img + ((size_t)yy * W + xx) * 3;
            const double gr = __dadd_rn(__dadd_rn(__dmul_rn(0.299, (double)px[0]),
                                                  __dmul_rn(0.587, (double)px[1])),
                                        __dmul_rn(0.114, (double)px[2]));
            s[t] = __dmul_rn((double)mask[t], gr);
        }
        __syncwarp();
        if (lane == 0) {
            double mu = 0.0;
            for (int t = 0; t < n; ++t) mu = __dadd_rn(mu, s[t]);
            s_ab[wib] = __ddiv_rn(mu, (double)n);
        }
        __syncwarp();
        const double mu = s_ab[wib];
        for (int t = lane; t < n; t += 32) s[t] = __dadd_rn(s[t], -mu);
        __syncwarp();
        if (lane == 0) {
            double ss = 0.0;
            for (int t = 0; t < n; ++t) ss = __dadd_rn(ss, __dmul_rn(s[t], s[t]));
            s_ab[wib] = ss;
        }
        __syncwarp();
        const double ss = s_ab[wib];
        if (ss == 0.0) {
            for (int t = lane; t < n; t += 32) s[t] = 0.0;
        } else {
            const double nrm = __dsqrt_rn(ss);
            for (int t = lane; t < n; t += 32) s[t] = __ddiv_rn(s[t], nrm);
        }
        __syncwarp();
        // codes: one lane per code index, each an index-order dot product
        const int jlo = g.y < 0 ? 0 : g.y, jhi = g.y < 0 ? k : g.y + 1;
        for (int j = jlo + lane; j < jhi; j += 32) {
            double a = 0.0;
            for (int t = 0; t < n; ++t)
                a = __dadd_rn(a, __dmul_rn((double)omega[(size_t)j * n + t], s[t]));
            if (fabs(a) <= tau) atomicOr(bitmask + (size_t)g.x * Wk + (j >> 5), 1u << (j & 31));
        }
        __syncwarp();
    }
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

cudaError_t launch_codes_f32(const CodesArgs& a, cudaStream_t st) {
    const int n = a.p * a.p;
    rownorm_kernel<<<(a.k + 127) / 128, 128, 0, st>>>(a.omega, a.k, n, a.rownorm, a.guard_count);
    cudaError_t e;
    switch (a.p) {
        case 3: e = launch_p<3>(a, st); break;
        case 5: e = launch_p<5>(a, st); break;
        case 7: e = launch_p<7>(a, st); break;
        case 9: e = launch_p<9>(a, st); break;
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    if (!a.bitmask) return cudaSuccess;
    codes_guard_kernel<<<152 * 4, 128, 0, st>>>(a.img, a.H, a.W, a.omega, a.k, a.mask, a.p, a.tau,
                                                a.guard, a.guard_cap, a.guard_count, a.bitmask,
                                                a.d_err);
    return cudaGetLastError();
}

cudaError_t launch_cosupport(const float* codes, long long P, int k, double tau,
                             uint32_t* bitmask, cudaStream_t st) {
    cosupport_kernel<<<152 * 8, 256, 0, st>>>(codes, P * k, k, tau, bitmask);
    return cudaGetLastError();
}
