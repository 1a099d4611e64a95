// Convex multilabel segmentation on the data term (Sec. 4): the relaxed
// energy of Eq. (energy1) / Eq. (sets) minimised by the primal-dual
// iteration of Eq. (algo), then binarised by argmax.
//
// Discretisation (the paper gives none): forward differences with a zero
// difference across the last row / column for grad, its negative adjoint for
// div; edge weight g(x) = exp(-|grad I(x)| / gamma) / (2 gamma) with |grad I|
// the Euclidean norm of the forward differences of the three channels of
// 255 I; step sizes by diagonal preconditioning: 1/2 for xi and mu, 1/5 for
// u, 1/|Omega| for m; start u = 1/n, m = 1, xi = mu = 0. Per iteration, three
// launches: the dual step (xi, mu and per-block sums of mu), the m step
// (fixed-order sums over the blocks), the primal step (u with Michelot's
// simplex projection per pixel, and the over-relaxed copies).
#include <cstdint>

#include "internal.h"

namespace {

constexpr int SB = 256;  // threads per block

__global__ void seg_bound_kernel(const float* __restrict__ img, int H, int W, float lam,
                                 float gamma, float* __restrict__ bound) {
    const long long P = (long long)H * W;
    for (long long q = blockIdx.x * (long long)SB + threadIdx.x; q < P;
         q += (long long)gridDim.x * SB) {
        const int y = (int)(q / W), x = (int)(q % W);
        float s = 0.f;
        for (int c = 0; c < 3; ++c) {
            const float v = 255.f * img[q * 3 + c];
            const float dx = x + 1 < W ? 255.f * img[(q + 1) * 3 + c] - v : 0.f;
            const float dy = y + 1 < H ? 255.f * img[(q + W) * 3 + c] - v : 0.f;
            s = fmaf(dx, dx, fmaf(dy, dy, s));
        }
        const float g = expf(-sqrtf(s) / gamma) / (2.f * gamma);
        bound[q] = 0.5f * lam * g;
    }
}

__global__ void seg_init_kernel(long long nP, float u0, float* __restrict__ u,
                                float* __restrict__ ub, float* __restrict__ px,
                                float* __restrict__ py, float* __restrict__ mu) {
    for (long long e = blockIdx.x * (long long)SB + threadIdx.x; e < nP;
         e += (long long)gridDim.x * SB) {
        u[e] = u0;
        ub[e] = u0;
        px[e] = 0.f;
        py[e] = 0.f;
        mu[e] = 0.f;
    }
}

// Dual step for label blockIdx.y: xi <- Pi_Kg(xi + 1/2 grad ub),
// mu <- min(0, mu + 1/2 (mb - ub)); per-block sums of the new mu.
__global__ void __launch_bounds__(SB) seg_dual_kernel(
    int H, int W, const float* __restrict__ ub, const float* __restrict__ mb,
    const float* __restrict__ bound, float* __restrict__ px, float* __restrict__ py,
    float* __restrict__ mu, float* __restrict__ parts) {
    __shared__ float red[SB / 32];
    const long long P = (long long)H * W;
    const int i = blockIdx.y;
    const float* ubi = ub + (size_t)i * P;
    float acc = 0.f;
    for (long long q = blockIdx.x * (long long)SB + threadIdx.x; q < P;
         q += (long long)gridDim.x * SB) {
        const int y = (int)(q / W), x = (int)(q % W);
        const float c = ubi[q];
        const float gx = x + 1 < W ? ubi[q + 1] - c : 0.f;
        const float gy = y + 1 < H ? ubi[q + W] - c : 0.f;
        const size_t e = (size_t)i * P + q;
        float ax = px[e] + 0.5f * gx, ay = py[e] + 0.5f * gy;
        const float b = bound[q];
        const float nrm = sqrtf(ax * ax + ay * ay);
        if (nrm > b) {
            const float sc = b > 0.f ? b / nrm : 0.f;
            ax *= sc;
            ay *= sc;
        }
        px[e] = ax;
        py[e] = ay;
        const float m = fminf(0.f, mu[e] + 0.5f * (mb[i] - c));
        mu[e] = m;
        acc += m;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.f;
        for (int w = 0; w < SB / 32; ++w) s += red[w];
        parts[(size_t)i * gridDim.x + blockIdx.x] = s;
    }
}

// m step: m <- clamp(m - (nu + sum mu) / |Omega|, 0, 1), mb = 2 m_new - m.
__global__ void seg_m_kernel(int n, int nblk, const float* __restrict__ parts, float nu,
                             float inv_area, float* __restrict__ m, float* __restrict__ mb) {
    const int i = threadIdx.x;
    if (i >= n) return;
    float s = 0.f;
    for (int b = 0; b < nblk; ++b) s += parts[(size_t)i * nblk + b];
    const float mn = fminf(1.f, fmaxf(0.f, m[i] - inv_area * (nu + s)));
    mb[i] = 2.f * mn - m[i];
    m[i] = mn;
}

// Primal step per pixel: u <- Pi_simplex(u - 1/5 (-div xi + f - mu)) by
// Michelot's algorithm over the labels, ub = 2 u_new - u.
__global__ void __launch_bounds__(SB) seg_primal_kernel(
    int H, int W, int n, const float* __restrict__ f, const float* __restrict__ px,
    const float* __restrict__ py, const float* __restrict__ mu, float* __restrict__ u,
    float* __restrict__ ub) {
    const long long P = (long long)H * W;
    for (long long q = blockIdx.x * (long long)SB + threadIdx.x; q < P;
         q += (long long)gridDim.x * SB) {
        const int y = (int)(q / W), x = (int)(q % W);
        float v[CS_MAX_LABELS];
        uint64_t active = n >= 64 ? ~0ull : ((1ull << n) - 1ull);
        for (int i = 0; i < n; ++i) {
            const size_t e = (size_t)i * P + q;
            float d = 0.f;  // div xi
            if (x + 1 < W) d += px[e];
            if (x > 0) d -= px[e - 1];
            if (y + 1 < H) d += py[e];
            if (y > 0) d -= py[e - W];
            v[i] = u[e] - 0.2f * (-d + f[e] - mu[e]);
        }
        // Michelot: project onto the active indices' hyperplane, drop negatives
        float shift = 0.f;
        for (int round = 0; round < n; ++round) {
            float s = 0.f;
            int cnt = 0;
            for (int i = 0; i < n; ++i)
                if ((active >> i) & 1ull) {
                    s += v[i];
                    ++cnt;
                }
            shift = (s - 1.f) / (float)cnt;
            uint64_t neg = 0;
            for (int i = 0; i < n; ++i)
                if (((active >> i) & 1ull) && v[i] - shift < 0.f) neg |= 1ull << i;
            if (!neg) break;
            active &= ~neg;
        }
        for (int i = 0; i < n; ++i) {
            const size_t e = (size_t)i * P + q;
            const float un = ((active >> i) & 1ull) ? v[i] - shift : 0.f;
            ub[e] = 2.f * un - u[e];
            u[e] = un;
        }
    }
}

__global__ void seg_minit_kernel(int n, float* __restrict__ m, float* __restrict__ mb) {
    if (threadIdx.x < n) m[threadIdx.x] = mb[threadIdx.x] = 1.f;
}

__global__ void seg_argmax_kernel(long long P, int n, const float* __restrict__ u,
                                  int32_t* __restrict__ labels) {
    for (long long q = blockIdx.x * (long long)SB + threadIdx.x; q < P;
         q += (long long)gridDim.x * SB) {
        int best = 0;
        float bv = u[q];
        for (int i = 1; i < n; ++i) {
            const float v = u[(size_t)i * P + q];
            if (v > bv) {
                bv = v;
                best = i;
            }
        }
        labels[q] = best;
    }
}

}  // namespace

size_t seg_scratch_bytes(long long P, int n, int nblk) {
    return sizeof(float) * ((size_t)4 * n * P + (size_t)P + (size_t)n * nblk + 4 * (size_t)n) + 1024;
}

cudaError_t launch_segment(const SegArgs& a, cudaStream_t st) {
    const long long P = (long long)a.H * a.W;
    const int n = a.n_labels;
    float* ub = a.scratch;
    float* px = ub + (size_t)n * P;
    float* py = px + (size_t)n * P;
    float* mu = py + (size_t)n * P;
    float* bound = mu + (size_t)n * P;
    float* parts = bound + P;
    float* m = parts + (size_t)n * a.nblk;
    float* mb = m + n;
    const int gP = (int)((P + SB - 1) / SB < 4096 ? (P + SB - 1) / SB : 4096);
    const long long nP = (long long)n * P;
    const int gnP = (int)((nP + SB - 1) / SB < 8192 ? (nP + SB - 1) / SB : 8192);
    seg_bound_kernel<<<gP, SB, 0, st>>>(a.img, a.H, a.W, a.lambda, a.gamma, bound);
    seg_init_kernel<<<gnP, SB, 0, st>>>(nP, 1.f / (float)n, a.u, ub, px, py, mu);
    seg_minit_kernel<<<1, 64, 0, st>>>(n, m, mb);
    for (int it = 0; it < a.iterations; ++it) {
        seg_dual_kernel<<<dim3(a.nblk, n), SB, 0, st>>>(a.H, a.W, ub, mb, bound, px, py, mu,
                                                         parts);
        seg_m_kernel<<<1, 64, 0, st>>>(n, a.nblk, parts, a.nu, 1.f / (float)P, m, mb);
        seg_primal_kernel<<<gP, SB, 0, st>>>(a.H, a.W, n, a.f, px, py, mu, a.u, ub);
    }
    if (a.labels) seg_argmax_kernel<<<gP, SB, 0, st>>>(P, n, a.u, a.labels);
    return cudaGetLastError();
}
