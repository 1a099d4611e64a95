// Smooth co-sparse texture (mode CS_MODE_SMOOTH): Sec. 2 Eq. (map_tsm)
// iota_sigma(a)_j = exp(-a_j^2 / sigma), Eq. (approx_cosupp) and Sec. 3.1
// c_i = elementwise median of the iota of label i's scribble samples, and
// Eq. (post_text) P(s_x, x | i) = softmax_i(-||c_i - iota(O s_x)||_1 / beta_i(x)),
// added to the Parzen colour-location log-likelihood of Eq. (joined).
//
// Codes here are FP32 dot products of the FP32-normalised patch (the
// arithmetic of the FP32 codes kernel: Kahan mean, reciprocal norm); a patch
// whose centred norm is within the FP32 bound of zero is taken as flat
// (s = 0, every code 0, iota = 1). Three launches after the sum:
//   smooth_iota_samples_kernel  iota of every scribble sample (code-major)
//   smooth_median_kernel        c_i by exact radix selection (one block per
//                               label and code; the mean of the two middle
//                               values for an even count)
//   smooth_texture_kernel       per pixel: iota, l1 to each c_i, the texture
//                               log-posterior added to -L, label posteriors
#include <cstdint>

#include "internal.h"

namespace {

constexpr int ST = 16;                 // pixel tile of the texture kernel: 16 x 16
constexpr int SL = 128;                // samples per block of the sample kernel
constexpr float SU32 = 5.9604645e-08f;  // 2^-24

__device__ __forceinline__ float gray_of(const float* px) {
    return __fadd_rn(__fadd_rn(__fmul_rn(0.299f, px[0]), __fmul_rn(0.587f, px[1])),
                     __fmul_rn(0.114f, px[2]));
}
__device__ __forceinline__ float gabs_of(const float* px) {
    return (0.299f * fabsf(px[0]) + 0.587f * fabsf(px[1]) + 0.114f * fabsf(px[2])) *
           (1.f + 4 * SU32);
}

// Normalised masked patch s (N values, padded to NP with zeros) from gray
// values g(t) and bounds ga(t) of window position t = dy P + dx.
template <int P, class GF, class AF>
__device__ __forceinline__ void norm_patch(const float* w, GF g, AF ga, float (&s)[(P * P + 3) & ~3]) {
    constexpr int N = P * P, NP = (N + 3) & ~3;
#pragma unroll
    for (int t = N; t < NP; ++t) s[t] = 0.f;
    float sum = 0.f, kc = 0.f, vabs = 0.f, e2 = 0.f;
#pragma unroll
    for (int t = 0; t < N; ++t) {
        const float v = __fmul_rn(w[t], g(t));
        s[t] = v;
        const float yk = __fsub_rn(v, kc);
        const float tk = __fadd_rn(sum, yk);
        kc = __fsub_rn(__fsub_rn(tk, sum), yk);
        sum = tk;
        vabs += fabsf(v);
        const float ew = fabsf(w[t]) * ga(t);
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
    const float dc = (2.f * 5.1f * SU32) * sqrtf(e2) * 1.0001f +
                     3.1f * SU32 * vabs * rsqrtf((float)N) * 1.0001f + SU32 * cn;
    const float inv = cn > 4.f * dc ? __frcp_rn(cn) : 0.f;  // flat: s = 0
#pragma unroll
    for (int t = 0; t < N; ++t) s[t] = __fmul_rn(s[t], inv);
}

// Loads rows j0 .. j0 + 31 of O into shared memory (NP floats per row).
template <int P>
__device__ __forceinline__ void load_rows(float* s_om, const float* omega, int k, int j0,
                                          int tid, int nthr) {
    constexpr int N = P * P, NP = (N + 3) & ~3;
    const int rows = min(32, k - j0);
    for (int i = tid; i < 32 * NP; i += nthr) {
        const int jj = i / NP, t = i % NP;
        s_om[i] = (jj < rows && t < N) ? omega[(size_t)(j0 + jj) * N + t] : 0.f;
    }
}

__device__ __forceinline__ float dot_row(const float* row, const float* s, int np4) {
    const float4* o4 = reinterpret_cast<const float4*>(row);
    float a0 = 0.f, a1 = 0.f;
    for (int t4 = 0; t4 < np4; ++t4) {
        const float4 o = o4[t4];
        a0 = fmaf(o.x, s[4 * t4 + 0], a0);
        a1 = fmaf(o.y, s[4 * t4 + 1], a1);
        a0 = fmaf(o.z, s[4 * t4 + 2], a0);
        a1 = fmaf(o.w, s[4 * t4 + 3], a1);
    }
    return a0 + a1;
}

// iota of every scribble sample (every pixel when sample_pix is null),
// code-major: iota_smp[j * S + s].
template <int P>
__global__ void __launch_bounds__(SL) smooth_iota_samples_kernel(
    const float* __restrict__ img, int H, int W, const float* __restrict__ omega, int k,
    const float* __restrict__ mask, const int32_t* __restrict__ sample_pix, int S, float sigma,
    float* __restrict__ iota_smp) {
    constexpr int N = P * P, NP = (N + 3) & ~3, R = (P - 1) / 2;
    __shared__ __align__(16) float s_om[32 * NP];
    __shared__ float s_w[N];
    for (int i = threadIdx.x; i < N; i += SL) s_w[i] = mask[i];
    __syncthreads();
    const int s_idx = blockIdx.x * SL + threadIdx.x;
    const bool live = s_idx < S;
    int pix = live ? (sample_pix ? sample_pix[s_idx] : s_idx) : 0;  // no list: every pixel
    if (pix < 0 || pix >= H * W) pix = 0;  // reported by the distance transform's seed pass
    const int y = pix / W, x = pix % W;
    auto px_at = [&](int t) {
        const int yy = min(max(y + t / P - R, 0), H - 1), xx = min(max(x + t % P - R, 0), W - 1);
        return img + ((size_t)yy * W + xx) * 3;
    };
    float s[NP];
    norm_patch<P>(s_w, [&](int t) { return gray_of(px_at(t)); },
                  [&](int t) { return gabs_of(px_at(t)); }, s);
    const float nsig = -1.f / sigma;
    for (int j0 = 0; j0 < k; j0 += 32) {
        __syncthreads();
        load_rows<P>(s_om, omega, k, j0, threadIdx.x, SL);
        __syncthreads();
        const int rows = min(32, k - j0);
        for (int jj = 0; jj < rows; ++jj) {
            const float a = dot_row(s_om + jj * NP, s, NP / 4);
            if (live) iota_smp[(size_t)(j0 + jj) * S + s_idx] = expf(a * a * nsig);
        }
    }
}

// Order-preserving map of a float's bits to an unsigned key, and back.
__device__ __forceinline__ unsigned f2key(float f) {
    const unsigned u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float key2f(unsigned k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// r-th smallest (0-based) of the m floats get(0 .. m-1) by four 8-bit radix
// passes over their order-preserving keys.
template <class Get>
__device__ float radix_select(Get get, int m, int r, unsigned* hist, unsigned* s_state) {
    unsigned prefix = 0, pmask = 0;
    for (int pass = 0; pass < 4; ++pass) {
        const int shift = 24 - 8 * pass;
        for (int b = threadIdx.x; b < 256; b += blockDim.x) hist[b] = 0;
        __syncthreads();
        for (int i = threadIdx.x; i < m; i += blockDim.x) {
            const unsigned u = f2key(get(i));
            if ((u & pmask) == prefix) atomicAdd(hist + ((u >> shift) & 255u), 1u);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned acc = 0;
            int d = 0;
            for (; d < 255; ++d) {
                if (acc + hist[d] > (unsigned)r) break;
                acc += hist[d];
            }
            s_state[0] = (unsigned)d;
            s_state[1] = (unsigned)r - acc;
        }
        __syncthreads();
        prefix |= s_state[0] << shift;
        pmask |= 255u << shift;
        r = (int)s_state[1];
        __syncthreads();
    }
    return key2f(prefix);
}

// c[i * k + j] = median over label i's samples of iota_smp[j][s].
__global__ void __launch_bounds__(256) smooth_median_kernel(
    const float* __restrict__ iota_smp, int S, int k, const int32_t* __restrict__ label_off,
    float* __restrict__ reps) {
    __shared__ unsigned hist[256];
    __shared__ unsigned s_state[2];
    const int i = blockIdx.y, j = blockIdx.x;
    const int off = label_off[i], m = label_off[i + 1] - off;
    const float* v = iota_smp + (size_t)j * S + off;
    auto get = [&](int e) { return v[e]; };
    const float lo = radix_select(get, m, (m - 1) / 2, hist, s_state);
    const float hi = (m % 2) ? lo : radix_select(get, m, m / 2, hist, s_state);
    if (threadIdx.x == 0) reps[(size_t)i * k + j] = (m % 2) ? lo : __fmul_rn(0.5f, __fadd_rn(lo, hi));
}

// Per pixel: iota of its codes, l1 to each representative, the texture
// log-posterior added to L (neglog holds -L of the Parzen sum), then the
// label posteriors.
template <int P>
__global__ void __launch_bounds__(ST * ST) smooth_texture_kernel(
    const float* __restrict__ img, int H, int W, const float* __restrict__ omega, int k,
    const float* __restrict__ mask, float sigma, const float* __restrict__ reps, int n_labels,
    const int32_t* __restrict__ dist2, float alpha, float d_min, float kappa_beta,
    float* __restrict__ neglog, float* __restrict__ post) {
    constexpr int N = P * P, NP = (N + 3) & ~3, R = (P - 1) / 2, TW = ST + P - 1;
    extern __shared__ __align__(16) float sm[];
    float* s_om = sm;                          // 32 x NP
    float* s_gray = s_om + 32 * NP;            // TW x TW
    float* s_gabs = s_gray + TW * TW;          // TW x TW
    float* s_w = s_gabs + TW * TW;             // N
    float* s_rep = s_w + ((N + 3) & ~3);       // n_labels x k
    float* s_acc = s_rep + (size_t)n_labels * k;  // n_labels x (ST * ST)
    const int tid = threadIdx.y * ST + threadIdx.x;
    const int y0 = blockIdx.y * ST, x0 = blockIdx.x * ST;
    for (int i = tid; i < TW * TW; i += ST * ST) {
        const int ly = i / TW, lx = i % TW;
        const int yy = min(max(y0 + ly - R, 0), H - 1), xx = min(max(x0 + lx - R, 0), W - 1);
        const float* px = img + ((size_t)yy * W + xx) * 3;
        s_gray[i] = gray_of(px);
        s_gabs[i] = gabs_of(px);
    }
    for (int i = tid; i < N; i += ST * ST) s_w[i] = mask[i];
    for (int i = tid; i < n_labels * k; i += ST * ST) s_rep[i] = reps[i];
    for (int i = 0; i < n_labels; ++i) s_acc[i * ST * ST + tid] = 0.f;
    __syncthreads();
    const int y = y0 + threadIdx.y, x = x0 + threadIdx.x;
    const bool live = y < H && x < W;
    float s[NP];
    norm_patch<P>(s_w,
                  [&](int t) { return s_gray[(threadIdx.y + t / P) * TW + threadIdx.x + t % P]; },
                  [&](int t) { return s_gabs[(threadIdx.y + t / P) * TW + threadIdx.x + t % P]; },
                  s);
    const float nsig = -1.f / sigma;
    for (int j0 = 0; j0 < k; j0 += 32) {
        __syncthreads();
        load_rows<P>(s_om, omega, k, j0, tid, ST * ST);
        __syncthreads();
        const int rows = min(32, k - j0);
        for (int jj = 0; jj < rows; ++jj) {
            const float a = dot_row(s_om + jj * NP, s, NP / 4);
            const float io = expf(a * a * nsig);
            for (int i = 0; i < n_labels; ++i)
                s_acc[i * ST * ST + tid] += fabsf(s_rep[(size_t)i * k + j0 + jj] - io);
        }
    }
    if (!live) return;
    const long long P_ = (long long)H * W;
    const int pix = y * W + x;
    // texture log-posterior, Eq. (post_text), beta_i = kappa_beta rho_i
    float tmax = -INFINITY;
    for (int i = 0; i < n_labels; ++i) {
        const float rho = alpha * fmaxf(sqrtf((float)dist2[(size_t)i * P_ + pix]), d_min);
        const float t = -s_acc[i * ST * ST + tid] / (kappa_beta * rho);
        s_acc[i * ST * ST + tid] = t;
        tmax = fmaxf(tmax, t);
    }
    float ts = 0.f;
    for (int i = 0; i < n_labels; ++i) ts += expf(s_acc[i * ST * ST + tid] - tmax);
    const float tl = tmax + logf(ts);
    float lmax = -INFINITY;
    for (int i = 0; i < n_labels; ++i) {
        const float L = -neglog[(size_t)i * P_ + pix] + s_acc[i * ST * ST + tid] - tl;
        s_acc[i * ST * ST + tid] = L;
        lmax = fmaxf(lmax, L);
    }
    float ls = 0.f;
    for (int i = 0; i < n_labels; ++i) ls += expf(s_acc[i * ST * ST + tid] - lmax);
    const float lse = lmax + logf(ls);
    for (int i = 0; i < n_labels; ++i) {
        const float L = s_acc[i * ST * ST + tid];
        neglog[(size_t)i * P_ + pix] = -L;
        if (post) post[(size_t)i * P_ + pix] = expf(L - lse);
    }
}

template <int P>
cudaError_t smooth_p(const SmoothArgs& a, cudaStream_t st) {
    constexpr int N = P * P, NP = (N + 3) & ~3, TW = ST + P - 1;
    smooth_iota_samples_kernel<P><<<(a.S + SL - 1) / SL, SL, 0, st>>>(
        a.img, a.H, a.W, a.omega, a.k, a.mask, a.sample_pix, a.S, a.sigma, a.iota_smp);
    smooth_median_kernel<<<dim3(a.k, a.n_labels), 256, 0, st>>>(a.iota_smp, a.S, a.k,
                                                                 a.d_label_off, a.reps);
    const size_t smem = sizeof(float) * ((size_t)32 * NP + 2 * TW * TW + ((N + 3) & ~3) +
                                         (size_t)a.n_labels * a.k + (size_t)a.n_labels * ST * ST);
    cudaError_t e = cudaFuncSetAttribute(smooth_texture_kernel<P>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grd((a.W + ST - 1) / ST, (a.H + ST - 1) / ST);
    smooth_texture_kernel<P><<<grd, dim3(ST, ST), smem, st>>>(
        a.img, a.H, a.W, a.omega, a.k, a.mask, a.sigma, a.reps, a.n_labels, a.dist2, a.alpha,
        a.d_min, a.kappa_beta, a.neglog, a.post);
    return cudaGetLastError();
}

template <int P>
cudaError_t iota_pixels_p(const float* img, int H, int W, const float* omega, int k,
                          const float* mask, float sigma, float* iota, cudaStream_t st) {
    const int S = H * W;
    smooth_iota_samples_kernel<P><<<(S + SL - 1) / SL, SL, 0, st>>>(img, H, W, omega, k, mask,
                                                                   nullptr, S, sigma, iota);
    return cudaGetLastError();
}

}  // namespace

size_t smooth_smem_bytes(int p, int k, int n_labels) {
    const int N = p * p, NP = (N + 3) & ~3, TW = ST + p - 1;
    return sizeof(float) * ((size_t)32 * NP + 2 * TW * TW + NP + (size_t)n_labels * k +
                            (size_t)n_labels * ST * ST);
}

cudaError_t launch_iota_pixels(const float* img, int H, int W, const float* omega, int k, int p,
                               const float* mask, float sigma, float* iota, cudaStream_t st) {
    switch (p) {
        case 3: return iota_pixels_p<3>(img, H, W, omega, k, mask, sigma, iota, st);
        case 5: return iota_pixels_p<5>(img, H, W, omega, k, mask, sigma, iota, st);
        case 7: return iota_pixels_p<7>(img, H, W, omega, k, mask, sigma, iota, st);
        case 9: return iota_pixels_p<9>(img, H, W, omega, k, mask, sigma, iota, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_smooth(const SmoothArgs& a, cudaStream_t st) {
    switch (a.p) {
        case 3: return smooth_p<3>(a, st);
        case 5: return smooth_p<5>(a, st);
        case 7: return smooth_p<7>(a, st);
        case 9: return smooth_p<9>(a, st);
        default: return cudaErrorInvalidValue;
    }
}
