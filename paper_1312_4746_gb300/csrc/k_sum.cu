// Pixel x sample likelihood sum, FP32 CUDA-core form (Sec. 3.1, Eq. color,
// Eq. post_text, Eq. joined, Eq. energy1).
//
// For pixel x and label i, with rho = alpha * max(sqrt(D_i(x)), d_min) and
// beta = kappa_beta * rho, every sample j of the label contributes
//   e_j = -|x - x_j|^2 / (2 rho^2) - |I(x) - I_j|^2 / (2 sigma_c2)
//         - w_t TSM(b_x, b_j) / beta            (w_t = 1 per-sample, 0 factorised)
// and L_i(x) = logsumexp_j e_j - log m_i - log(2 pi rho^2) - 1.5 log(2 pi sigma_c2).
// The factorised form adds the texture log-posterior of Eq. (post_text) with
// the label's majority co-support. Posteriors are the softmax of L over
// labels; the data term is f_i = -L_i.
//
// Layout: one block of 128 threads owns NPIX * 128 consecutive pixels (pixel
// q = base + u * 128 + tid, u < NPIX); it loops over the labels and streams
// each label's samples through shared memory in tiles of 128 (SoA, padded
// with a far-away location so padded terms vanish). Exponents are in log2
// units; the log-sum-exp is online with a running maximum per 16-sample
// chunk and a TwoSum-compensated running sum. Distances are exact integers
// carried in FP32 (coordinates < 2^24), the TSM is popc over XORed words.
#include <cstdint>

#include "internal.h"

namespace {

constexpr int THREADS = 128;
constexpr int TS = 128;  // samples per shared-memory tile
constexpr int CH = 16;   // samples per online-max chunk
constexpr float LOG2E = 1.4426950408889634f;
constexpr float LN2 = 0.6931471805599453f;
constexpr float FAR = 1.0e18f;

__device__ __forceinline__ float ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// rho, -log2(e)/(2 s2), -w log2(e)/beta and the location variance s2
// (rho^2, or rho itself when rho is read as the variance)
__device__ __forceinline__ void label_consts(int D, float alpha, float d_min, float kappa_beta,
                                             bool rho_var, float& rho, float& nA, float& nB) {
    float d = sqrtf((float)D);
    rho = alpha * fmaxf(d, d_min);
    nA = -LOG2E / (2.f * (rho_var ? rho : rho * rho));
    nB = -LOG2E / (kappa_beta * rho);
}

template <int WK, int NPIX>
__global__ void __launch_bounds__(THREADS) sum_plain_kernel(SumArgs a) {
    __shared__ float s_x[TS], s_y[TS], s_r[TS], s_g[TS], s_b[TS];
    __shared__ uint32_t s_bits[WK][TS];

    const long long P = (long long)a.H * a.W;
    const int tid = threadIdx.x;
    const float nC = -LOG2E / (2.f * a.sigma_c2);
    const float log_col_norm = 1.5f * logf(6.283185307179586f * a.sigma_c2);
    const float wtex = a.mode == CS_MODE_PERSAMPLE ? 1.f : 0.f;
    // work items: every pixel, or the pixels of a device list (count on the device)
    const long long n_items = a.pix_list ? (long long)min(*a.list_count, a.list_cap) : P;

    for (long long base = (long long)blockIdx.x * THREADS * NPIX; base < n_items;
         base += (long long)gridDim.x * THREADS * NPIX) {
    float px[NPIX], py[NPIX], pr[NPIX], pg[NPIX], pb[NPIX];
    uint32_t pbits[NPIX][WK];
    bool live[NPIX];
    long long qpix[NPIX], item[NPIX];
#pragma unroll
    for (int u = 0; u < NPIX; ++u) {
        item[u] = base + u * THREADS + tid;
        live[u] = item[u] < n_items;
        long long qq = live[u] ? (a.pix_list ? (long long)a.pix_list[item[u]] : item[u]) : 0;
        qpix[u] = qq;
        px[u] = (float)(qq % a.W);
        py[u] = (float)(qq / a.W);
        pr[u] = a.img[qq * 3 + 0];
        pg[u] = a.img[qq * 3 + 1];
        pb[u] = a.img[qq * 3 + 2];
#pragma unroll
        for (int w = 0; w < WK; ++w) pbits[u][w] = a.bitmask[qq * WK + w];
    }

    for (int i = 0; i < a.n_labels; ++i) {
        const int off0 = a.d_label_off[i], off1 = a.d_label_off[i + 1];
        float nA[NPIX], nB[NPIX], rho[NPIX], M[NPIX], S[NPIX], Cc[NPIX];
#pragma unroll
        for (int u = 0; u < NPIX; ++u) {
            long long q = qpix[u];
            label_consts(a.dist2[(size_t)i * P + q], a.alpha, a.d_min, a.kappa_beta, a.rho_var, rho[u],
                         nA[u], nB[u]);
            nB[u] *= wtex;
            M[u] = -INFINITY;
            S[u] = 0.f;
            Cc[u] = 0.f;
        }
        for (int t0 = off0; t0 < off1; t0 += TS) {
            const int nvalid = min(TS, off1 - t0);
            __syncthreads();
            {
                const int s = t0 + tid;
                const bool ok = tid < nvalid;
                s_x[tid] = ok ? a.t.sx[s] : FAR;
                s_y[tid] = ok ? a.t.sy[s] : 0.f;
                s_r[tid] = ok ? a.t.sr[s] : 0.f;
                s_g[tid] = ok ? a.t.sg[s] : 0.f;
                s_b[tid] = ok ? a.t.sb[s] : 0.f;
#pragma unroll
                for (int w = 0; w < WK; ++w)
                    s_bits[w][tid] = ok ? a.t.sbits[(size_t)w * a.n_samples + s] : 0u;
            }
            __syncthreads();
            const int nch = (nvalid + CH - 1) / CH;
            for (int c0 = 0; c0 < nch * CH; c0 += CH) {
                float e[NPIX][CH];
#pragma unroll
                for (int c = 0; c < CH; ++c) {
                    const int j = c0 + c;
                    const float sx = s_x[j], sy = s_y[j], sr = s_r[j], sg = s_g[j], sb = s_b[j];
                    uint32_t sbw[WK];
#pragma unroll
                    for (int w = 0; w < WK; ++w) sbw[w] = s_bits[w][j];
#pragma unroll
                    for (int u = 0; u < NPIX; ++u) {
                        const float dx = px[u] - sx, dy = py[u] - sy;
                        const float d2 = fmaf(dx, dx, dy * dy);
                        const float dr = pr[u] - sr, dg = pg[u] - sg, db = pb[u] - sb;
                        const float c2 = fmaf(dr, dr, fmaf(dg, dg, db * db));
                        int h = 0;
#pragma unroll
                        for (int w = 0; w < WK; ++w) h += __popc(pbits[u][w] ^ sbw[w]);
                        e[u][c] = fmaf(nA[u], d2, fmaf(nC, c2, nB[u] * (float)h));
                    }
                }
#pragma unroll
                for (int u = 0; u < NPIX; ++u) {
                    float m = e[u][0];
#pragma unroll
                    for (int c = 1; c < CH; ++c) m = fmaxf(m, e[u][c]);
                    if (m > M[u]) {
                        const float sc = ex2(M[u] - m);
                        S[u] *= sc;
                        Cc[u] *= sc;
                        M[u] = m;
                    }
                    float tsum = 0.f;
#pragma unroll
                    for (int c = 0; c < CH; ++c) tsum += ex2(e[u][c] - M[u]);
                    // TwoSum: S + tsum = s + err exactly
                    const float s = S[u] + tsum;
                    const float bb = s - S[u];
                    const float err = (S[u] - (s - bb)) + (tsum - bb);
                    S[u] = s;
                    Cc[u] += err;
                }
            }
        }
        const float logm = logf((float)(off1 - off0));
#pragma unroll
        for (int u = 0; u < NPIX; ++u) {
            if (!live[u]) continue;
            const long long q = qpix[u];
            const float lse = (M[u] + log2f(S[u] + Cc[u])) * LN2;
            if (a.T_out) {  // log kernel sum only (surrogate targets), compact layout
                a.T_out[(size_t)i * a.list_cap + item[u]] = lse;
                continue;
            }
            const float s2 = a.rho_var ? rho[u] : rho[u] * rho[u];
            const float L = lse - logm - logf(6.283185307179586f * s2) - log_col_norm;
            a.neglog[(size_t)i * P + q] = -L;
        }
    }
    if (a.T_out) continue;

    // label normalisation (and the factorised texture posterior)
#pragma unroll
    for (int u = 0; u < NPIX; ++u) {
        if (!live[u]) continue;
        const long long q = qpix[u];
        if (a.mode == CS_MODE_FACTORISED) {
            float tmax = -INFINITY;
            for (int i = 0; i < a.n_labels; ++i) {
                float rho, nA, nB;
                label_consts(a.dist2[(size_t)i * P + q], a.alpha, a.d_min, a.kappa_beta, a.rho_var, rho, nA, nB);
                int h = 0;
#pragma unroll
                for (int w = 0; w < WK; ++w) h += __popc(pbits[u][w] ^ a.t.rep[i * WK + w]);
                tmax = fmaxf(tmax, nB * (float)h);
            }
            float ts = 0.f;
            for (int i = 0; i < a.n_labels; ++i) {
                float rho, nA, nB;
                label_consts(a.dist2[(size_t)i * P + q], a.alpha, a.d_min, a.kappa_beta, a.rho_var, rho, nA, nB);
                int h = 0;
#pragma unroll
                for (int w = 0; w < WK; ++w) h += __popc(pbits[u][w] ^ a.t.rep[i * WK + w]);
                ts += ex2(nB * (float)h - tmax);
            }
            const float tlse2 = tmax + log2f(ts);
            for (int i = 0; i < a.n_labels; ++i) {
                float rho, nA, nB;
                label_consts(a.dist2[(size_t)i * P + q], a.alpha, a.d_min, a.kappa_beta, a.rho_var, rho, nA, nB);
                int h = 0;
#pragma unroll
                for (int w = 0; w < WK; ++w) h += __popc(pbits[u][w] ^ a.t.rep[i * WK + w]);
                // texture log-posterior, natural log
                a.neglog[(size_t)i * P + q] -= (nB * (float)h - tlse2) * LN2;
            }
        }
        float lmax = -INFINITY;
        for (int i = 0; i < a.n_labels; ++i) lmax = fmaxf(lmax, -a.neglog[(size_t)i * P + q]);
        float ls = 0.f;
        for (int i = 0; i < a.n_labels; ++i) ls += expf(-a.neglog[(size_t)i * P + q] - lmax);
        const float lse = lmax + logf(ls);
        if (a.post)
            for (int i = 0; i < a.n_labels; ++i)
                a.post[(size_t)i * P + q] = expf(-a.neglog[(size_t)i * P + q] - lse);
    }
    }  // work-item tiles
}

template <int WK>
cudaError_t launch_wk(const SumArgs& a, cudaStream_t st) {
    constexpr int NPIX = 1;
    const long long n = a.pix_list ? (long long)a.list_cap : (long long)a.H * a.W;
    long long blocks = (n + THREADS * NPIX - 1) / (THREADS * NPIX);
    if (a.pix_list && blocks > 152 * 16) blocks = 152 * 16;  // grid-stride over the list
    if (blocks < 1) blocks = 1;
    sum_plain_kernel<WK, NPIX><<<(unsigned)blocks, THREADS, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_sum_plain(const SumArgs& a, cudaStream_t st) {
    switch (a.Wk) {
        case 1: return launch_wk<1>(a, st);
        case 2: return launch_wk<2>(a, st);
        case 3: return launch_wk<3>(a, st);
        case 4: return launch_wk<4>(a, st);
        case 5: return launch_wk<5>(a, st);
        case 6: return launch_wk<6>(a, st);
        case 7: return launch_wk<7>(a, st);
        case 8: return launch_wk<8>(a, st);
        default: return cudaErrorInvalidValue;
    }
}
