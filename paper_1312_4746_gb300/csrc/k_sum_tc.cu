// Pixel x sample likelihood sum on the tensor cores (tcgen05), the fast form
// of Sec. 3.1 Eq. (color) x Eq. (post_text) (per-sample or factorised).
//
// Per pixel x and label i (log2 units, C = log2(e) / (2 sigma_c2),
// Bt = log2(e) / beta_i(x), nA = -log2(e) / (2 rho_i(x)^2)):
//   e_j = nA |x - x_j|^2 - C |I - I_j|^2 - Bt TSM(b_x, b_j)
//       = [Bt D1_j + nA |x - x_j|^2] + R0,   R0 = -Bt |b_x| - C |I|^2,
//   D1_j = sum_t (2 b_x,t - 1) b_j,t  +  (1/Bt) (2 C I.I_j - C |I_j|^2).
// The first sum is an exact integer (2 b_x.b_j - |b_j|, so TSM = |b_x| - it)
// from an FP8 (e4m3, values 0 and +-1) or BF16 MMA; the colour part is a
// 16-wide BF16 MMA over hi/lo splits of both factors (relative error about
// 2^-17), accumulated into the same FP32 tensor-memory accumulator. The
// location term is an exact integer difference on the CUDA cores. In the
// factorised form D1_j is the colour part with Bt = 1 and no texture MMA.
//
// One persistent CTA per SM; each pixel tile is 128 consecutive pixels (one
// TMEM lane each) and each sample tile 128 samples (one TMEM column each).
//   warp 16      TMA producer: bulk-copies pre-laid-out sample tiles (texture
//                slabs, colour slab, sample coordinates) into a 3-stage ring
//   warp 17      MMA issuer: texture slabs + colour slab -> TMEM buffer b
//                (double-buffered, 2 x 128 columns), commits to barriers
//   warps 0..15  epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31 and the
//                32 columns 32 (w / 4) .. +31 of each tile, keeps an online
//                log-sum-exp (lazy rescale, TwoSum-compensated sum), merges
//                the four column quarters per label, and finally normalises
//                over labels.
// Every mbarrier wait is bounded by the global timer; on expiry the CTA sets
// the device error word, stops issuing, drains its copies and MMAs, frees its
// tensor memory and exits.
#include <cuda_bf16.h>

#include <cstdint>
#include <vector>

#include "internal.h"
#include "tc_ptx.cuh"

namespace {

constexpr int BM = 128, BN = 128;
constexpr int STAGES = 3;
constexpr int EPQ = 4;                 // epilogue warps per TMEM lane quadrant
constexpr int EPI_WARPS = 4 * EPQ;     // 16
constexpr int CPW = BN / EPQ;          // columns per epilogue warp per tile (32)
constexpr int PRODUCER = EPI_WARPS;    // warp 16
constexpr int MMA_WARP = EPI_WARPS + 1;
constexpr int THREADS = (EPI_WARPS + 2) * 32;
constexpr uint32_t TMEM_COLS = 256;
constexpr float LOG2E = 1.4426950408889634f;
constexpr float LN2 = 0.6931471805599453f;
constexpr uint64_t WAIT_NS = 1000000000ull;  // 1 s per wait
constexpr float LAZY = 8.f;                  // rescale once the max grows by 2^8

struct TcArgs {
    const float* img;
    int H, W;
    const uint32_t* bitmask;
    int k, Wk;
    int n_labels;
    const int32_t* d_label_off;
    const int32_t* d_tile_off;  // first sample tile of each label, n_labels + 1
    const uint8_t* blob;        // total_tiles * stage_bytes, laid out as a ring stage
    const uint32_t* rep;        // majority co-supports (factorised form)
    const int32_t* dist2;
    float alpha, d_min, kappa_beta, sigma_c2;
    float* neglog;
    float* post;
    int* d_err;
    int n_ptiles;
};

template <bool TEX8, int KS, bool PERSAMPLE>
struct Cfg {
    static constexpr int tex_bytes = PERSAMPLE ? KS * 4096 : 0;
    static constexpr int col_off = tex_bytes;
    static constexpr int xy_off = tex_bytes + 4096;
    static constexpr int stage_bytes = tex_bytes + 4096 + BN * 8;
    // shared memory map
    static constexpr int ring_off = 0;
    static constexpr int atex_off = ring_off + STAGES * stage_bytes;
    static constexpr int acol_off = atex_off + tex_bytes;
    static constexpr int xchg_off = acol_off + 2 * 4096;              // [4][EPQ-1][4][32] float4
    static constexpr int ls_off = xchg_off + 4 * (EPQ - 1) * 4 * 32 * 16;  // [64 labels][128] float
    static constexpr int bar_off = ls_off + CS_MAX_LABELS * BM * 4;
    static constexpr int n_bars = 3 * STAGES + 2 + 2 + 2 + 2 + 2 + 16;
    static constexpr int misc_off = bar_off + n_bars * 8;
    static constexpr int smem_bytes = misc_off + 16;
    static constexpr uint32_t id_tex = TEX8 ? tc::idesc(BM, BN, 0, 0) : tc::idesc(BM, BN, 1, 1);
    static constexpr uint32_t id_col = tc::idesc(BM, BN, 1, 1);
};

__device__ __forceinline__ float ex2f(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ uint16_t bf16_bits(float v) {
    return __bfloat16_as_ushort(__float2bfloat16_rn(v));
}
// v ~ hi + lo, both bf16, |v - hi - lo| <= 2^-18 |v|
__device__ __forceinline__ void split_bf16(float v, uint16_t& hi, uint16_t& lo) {
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    hi = __bfloat16_as_ushort(h);
    lo = bf16_bits(v - __bfloat162float(h));
}

__device__ __forceinline__ void set_abort(volatile int* abort_flag, int* d_err, int site) {
    *abort_flag = 1;
    if (atomicCAS(d_err, 0, CS_DEVERR_TIMEOUT) == 0) d_err[1] = site;
}

__device__ __forceinline__ bool wait_bar(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                         int* d_err, int site) {
    if (*abort_flag) return false;
    if (tc::mbar_wait(bar, parity, tc::globaltimer() + WAIT_NS)) return true;
    set_abort(abort_flag, d_err, site);
    return false;
}

// sample tiles of label i
__device__ __forceinline__ int tiles_of(const int32_t* tile_off, int i) {
    return tile_off[i + 1] - tile_off[i];
}

template <bool TEX8, int KS, bool PERSAMPLE>
__global__ void __launch_bounds__(THREADS, 1) sum_tc_kernel(TcArgs a) {
    using C = Cfg<TEX8, KS, PERSAMPLE>;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t* ring = smem + C::ring_off;
    uint8_t* atex = smem + C::atex_off;
    uint8_t* acol = smem + C::acol_off;
    float4* xchg = reinterpret_cast<float4*>(smem + C::xchg_off);
    float* Ls = reinterpret_cast<float*>(smem + C::ls_off);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + C::bar_off);
    uint64_t* full = bars;                      // [STAGES] tx-counted
    uint64_t* empty_mma = bars + STAGES;        // [STAGES] MMA commit
    uint64_t* empty_epi = bars + 2 * STAGES;    // [STAGES] epilogue warps
    uint64_t* tmem_full = bars + 3 * STAGES;    // [2] MMA commit
    uint64_t* tmem_empty = tmem_full + 2;       // [2] epilogue warps
    uint64_t* acol_full = tmem_full + 4;        // [2] epilogue warps
    uint64_t* acol_empty = tmem_full + 6;       // [2] MMA commit
    uint64_t* atex_full = tmem_full + 8;        // [1] epilogue warps
    uint64_t* atex_empty = tmem_full + 9;       // [1] MMA commit
    uint64_t* xchg_full = tmem_full + 10;       // [4 buffers][4 quadrants] column quarters 1..3
    uint32_t* tmem_base_s = reinterpret_cast<uint32_t*>(smem + C::misc_off);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + C::misc_off + 4);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long P = (long long)a.H * a.W;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            tc::mbar_init(full + s, 1);
            tc::mbar_init(empty_mma + s, 1);
            tc::mbar_init(empty_epi + s, EPI_WARPS);
        }
        for (int b = 0; b < 2; ++b) {
            tc::mbar_init(tmem_full + b, 1);
            tc::mbar_init(tmem_empty + b, EPI_WARPS);
            tc::mbar_init(acol_full + b, EPI_WARPS);
            tc::mbar_init(acol_empty + b, 1);
        }
        tc::mbar_init(atex_full, EPI_WARPS);
        tc::mbar_init(atex_empty, 1);
        for (int x = 0; x < 16; ++x) tc::mbar_init(xchg_full + x, EPQ - 1);
        *abort_flag = 0;
        tc::fence_mbar_init();
    }
    if (warp == 0) {
        tc::tmem_alloc(tmem_base_s, TMEM_COLS);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_base_s;

    if (warp == PRODUCER) {
        // ------------------------------------------------------------ TMA producer
        if (lane == 0) {
            long long it = 0;
            bool ok = true;
            for (int pt = blockIdx.x; ok && pt < a.n_ptiles; pt += gridDim.x)
                for (int i = 0; ok && i < a.n_labels; ++i) {
                    const int t0 = a.d_tile_off[i], nt = tiles_of(a.d_tile_off, i);
                    for (int t = 0; ok && t < nt; ++t, ++it) {
                        const int s = (int)(it % STAGES);
                        const uint32_t ph = (uint32_t)((it / STAGES) & 1);
                        ok = wait_bar(empty_mma + s, ph ^ 1, abort_flag, a.d_err, 1) &&
                             wait_bar(empty_epi + s, ph ^ 1, abort_flag, a.d_err, 2);
                        if (!ok) break;
                        tc::mbar_arrive_expect_tx(full + s, C::stage_bytes);
                        tc::bulk_g2s(ring + s * C::stage_bytes,
                                     a.blob + (size_t)(t0 + t) * C::stage_bytes, C::stage_bytes,
                                     full + s);
                    }
                }
            // drain: copies still in flight must land before the CTA exits
            for (long long d = (it > STAGES ? it - STAGES : 0); d < it; ++d)
                tc::mbar_wait(full + (int)(d % STAGES), (uint32_t)((d / STAGES) & 1),
                              tc::globaltimer() + WAIT_NS);
        }
    } else if (warp == MMA_WARP) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            long long it = 0, li = 0, lpt = 0;
            bool ok = true;
            long long last_b = -1;
            for (int pt = blockIdx.x; ok && pt < a.n_ptiles; pt += gridDim.x, ++lpt) {
                ok = wait_bar(atex_full, (uint32_t)(lpt & 1), abort_flag, a.d_err, 3);
                for (int i = 0; ok && i < a.n_labels; ++i, ++li) {
                    const int cb = (int)(li & 1);
                    ok = wait_bar(acol_full + cb, (uint32_t)((li >> 1) & 1), abort_flag, a.d_err, 4);
                    const int nt = tiles_of(a.d_tile_off, i);
                    for (int t = 0; ok && t < nt; ++t, ++it) {
                        const int s = (int)(it % STAGES), b = (int)(it & 1);
                        ok = wait_bar(full + s, (uint32_t)((it / STAGES) & 1), abort_flag, a.d_err, 5) &&
                             wait_bar(tmem_empty + b, (uint32_t)(((it >> 1) & 1) ^ 1), abort_flag,
                                      a.d_err, 6);
                        if (!ok) break;
                        tc::fence_after_sync();
                        const uint32_t d = tmem + (uint32_t)(b * BN);
                        const uint8_t* st = ring + s * C::stage_bytes;
                        if (PERSAMPLE) {
#pragma unroll
                            for (int sl = 0; sl < KS; ++sl) {
                                if (TEX8)
                                    tc::mma_fp8(d, tc::smem_desc(atex + sl * 4096),
                                                tc::smem_desc(st + sl * 4096), C::id_tex, sl > 0);
                                else
                                    tc::mma_bf16(d, tc::smem_desc(atex + sl * 4096),
                                                 tc::smem_desc(st + sl * 4096), C::id_tex, sl > 0);
                            }
                        }
                        tc::mma_bf16(d, tc::smem_desc(acol + cb * 4096),
                                     tc::smem_desc(st + C::col_off), C::id_col, PERSAMPLE ? 1 : 0);
                        tc::mma_commit(empty_mma + s);
                        tc::mma_commit(tmem_full + b);
                        last_b = it;
                    }
                    if (ok) tc::mma_commit(acol_empty + cb);
                }
                if (ok) tc::mma_commit(atex_empty);
            }
            // drain: the last MMAs must finish before the tensor memory is freed
            if (last_b >= 0)
                tc::mbar_wait(tmem_full + (int)(last_b & 1), (uint32_t)((last_b >> 1) & 1),
                              tc::globaltimer() + WAIT_NS);
        }
    } else {
        // ------------------------------------------------------------ epilogue
        const int q = warp & 3, hf = warp >> 2;  // lane quadrant, column quarter
        const int r = 32 * q + lane;             // pixel row of the tile
        const float Cc = LOG2E / (2.f * a.sigma_c2);
        const float log_col_norm = 1.5f * logf(6.283185307179586f * a.sigma_c2);
        long long it = 0, li = 0, lpt = 0;
        bool ok = true;
        for (int pt = blockIdx.x; ok && pt < a.n_ptiles; pt += gridDim.x, ++lpt) {
            const long long pix = (long long)pt * BM + r;
            const bool live = pix < P;
            const long long pq = live ? pix : 0;
            const float px = (float)(pq % a.W), py = (float)(pq / a.W);
            const float IR = a.img[pq * 3 + 0], IG = a.img[pq * 3 + 1], IB = a.img[pq * 3 + 2];
            const float I2 = fmaf(IR, IR, fmaf(IG, IG, IB * IB));
            uint32_t bx[8];
            int popx = 0;
#pragma unroll
            for (int w = 0; w < 8; ++w) {
                bx[w] = (w < a.Wk && live) ? a.bitmask[pq * a.Wk + w] : 0u;
                popx += __popc(bx[w]);
            }
            // texture operand rows: this warp writes slabs sl = hf, hf + EPQ, ...
            if (PERSAMPLE) {
                ok = wait_bar(atex_empty, (uint32_t)((lpt & 1) ^ 1), abort_flag, a.d_err, 7);
                if (!ok) break;
                for (int sl = hf; sl < KS; sl += EPQ) {
                    uint32_t wv[8];
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        uint32_t word = 0;
                        if (TEX8) {
                            // 4 fp8 values per 32-bit word: codes j = 32 sl + 4c .. +3
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                const int j = 32 * sl + 4 * c + e;
                                uint32_t v = 0;
                                if (live && j < a.k) v = ((bx[j >> 5] >> (j & 31)) & 1u) ? 0x38u : 0xB8u;
                                word |= v << (8 * e);
                            }
                        } else {
                            // 2 bf16 values per word: codes j = 16 sl + 2c .. +1
#pragma unroll
                            for (int e = 0; e < 2; ++e) {
                                const int j = 16 * sl + 2 * c + e;
                                uint32_t v = 0;
                                if (live && j < a.k) v = ((bx[j >> 5] >> (j & 31)) & 1u) ? 0x3F80u : 0xBF80u;
                                word |= v << (16 * e);
                            }
                        }
                        wv[c] = word;
                    }
                    uint8_t* base = atex + sl * 4096;
                    *reinterpret_cast<uint4*>(base + tc::slab_off(r, 0)) = make_uint4(wv[0], wv[1], wv[2], wv[3]);
                    *reinterpret_cast<uint4*>(base + tc::slab_off(r, 16)) = make_uint4(wv[4], wv[5], wv[6], wv[7]);
                }
                tc::fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(atex_full);
            } else if (lane == 0) {
                tc::mbar_arrive(atex_full);
            }

            for (int i = 0; ok && i < a.n_labels; ++i, ++li) {
                const int D = live ? a.dist2[(size_t)i * P + pq] : 0;
                const float rho = a.alpha * fmaxf(sqrtf((float)D), a.d_min);
                const float nA = -LOG2E / (2.f * rho * rho);
                const float Bt = PERSAMPLE ? LOG2E / (a.kappa_beta * rho) : 1.f;
                const float g = PERSAMPLE ? (a.kappa_beta * rho) / LOG2E : 1.f;
                // colour operand row (16 bf16): this warp writes half hf (hf < 2)
                const int cb = (int)(li & 1);
                ok = wait_bar(acol_empty + cb, (uint32_t)(((li >> 1) & 1) ^ 1), abort_flag, a.d_err, 8);
                if (!ok) break;
                if (hf < 2) {
                    uint16_t v[8];
                    if (hf == 0) {
                        uint16_t h0, l0, h1, l1;
                        split_bf16(2.f * Cc * g * IR, h0, l0);
                        split_bf16(2.f * Cc * g * IG, h1, l1);
                        v[0] = h0; v[1] = h0; v[2] = l0; v[3] = l0;
                        v[4] = h1; v[5] = h1; v[6] = l1; v[7] = l1;
                    } else {
                        uint16_t h2, l2, hg, lg;
                        split_bf16(2.f * Cc * g * IB, h2, l2);
                        split_bf16(g, hg, lg);
                        v[0] = h2; v[1] = h2; v[2] = l2; v[3] = l2;
                        v[4] = hg; v[5] = hg; v[6] = lg; v[7] = lg;
                    }
                    uint4 pk;
                    pk.x = v[0] | ((uint32_t)v[1] << 16);
                    pk.y = v[2] | ((uint32_t)v[3] << 16);
                    pk.z = v[4] | ((uint32_t)v[5] << 16);
                    pk.w = v[6] | ((uint32_t)v[7] << 16);
                    if (!live) pk = make_uint4(0, 0, 0, 0);
                    *reinterpret_cast<uint4*>(acol + cb * 4096 + tc::slab_off(r, 16 * hf)) = pk;
                    tc::fence_proxy_async_smem();
                }
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(acol_full + cb);

                const int m_i = a.d_label_off[i + 1] - a.d_label_off[i];
                const int nt = tiles_of(a.d_tile_off, i);
                float M = -INFINITY, S = 0.f, Ccomp = 0.f;
                for (int t = 0; t < nt; ++t, ++it) {
                    const int s = (int)(it % STAGES), b = (int)(it & 1);
                    ok = wait_bar(full + s, (uint32_t)((it / STAGES) & 1), abort_flag, a.d_err, 9) &&
                         wait_bar(tmem_full + b, (uint32_t)((it >> 1) & 1), abort_flag, a.d_err, 10);
                    if (!ok) break;
                    tc::fence_after_sync();
                    const int nvalid = min(BN, m_i - t * BN);
                    const float2* xy = reinterpret_cast<const float2*>(ring + s * C::stage_bytes + C::xy_off);
#pragma unroll
                    for (int c = 0; c < CPW / 16; ++c) {
                        const int col0 = hf * CPW + 16 * c;
                        uint32_t rv[16];
                        tc::tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * BN + col0), rv);
                        float e[16];
                        tc::tmem_ld_wait();
                        if (col0 < nvalid) {
                            float m = -INFINITY;
#pragma unroll
                            for (int u = 0; u < 16; ++u) {
                                const float2 sxy = xy[col0 + u];
                                const float dx = px - sxy.x, dy = py - sxy.y;
                                const float d2 = fmaf(dx, dx, dy * dy);
                                float v = fmaf(nA, d2, Bt * __uint_as_float(rv[u]));
                                v = (col0 + u < nvalid) ? v : -INFINITY;
                                e[u] = v;
                                m = fmaxf(m, v);
                            }
                            if (m > M + LAZY) {
                                const float sc = ex2f(M - m);
                                S *= sc;
                                Ccomp *= sc;
                                M = m;
                            }
                            float ts = 0.f;
#pragma unroll
                            for (int u = 0; u < 16; ++u) ts += ex2f(e[u] - M);
                            const float sn = S + ts;
                            const float bb = sn - S;
                            Ccomp += (S - (sn - bb)) + (ts - bb);
                            S = sn;
                        }
                    }
                    tc::fence_before_sync();
                    __syncwarp();
                    if (lane == 0) {
                        tc::mbar_arrive(tmem_empty + b);
                        tc::mbar_arrive(empty_epi + s);
                    }
                }
                if (!ok) break;
                // merge the EPQ column quarters of each pixel. Four exchange
                // buffers: a quarter can run at most two sample tiles ahead of
                // another (tensor memory is double-buffered and every label has
                // at least one tile), so buffer li & 3 is free when rewritten.
                const int xbuf = (int)(li & 3);
                float4* xb = xchg + (size_t)xbuf * (EPQ - 1) * 4 * 32;
                uint64_t* xbar = xchg_full + xbuf * 4 + q;
                if (hf > 0) {
                    xb[((hf - 1) * 4 + q) * 32 + lane] = make_float4(M, S, Ccomp, 0.f);
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(xbar);
                } else {
                    ok = wait_bar(xbar, (uint32_t)((li >> 2) & 1), abort_flag, a.d_err, 11);
                    if (!ok) break;
                    float Mm = M;
#pragma unroll
                    for (int h = 0; h < EPQ - 1; ++h) Mm = fmaxf(Mm, xb[(h * 4 + q) * 32 + lane].x);
                    float Sm = S * ex2f(M - Mm), Cm = Ccomp * ex2f(M - Mm);
#pragma unroll
                    for (int h = 0; h < EPQ - 1; ++h) {
                        const float4 v = xb[(h * 4 + q) * 32 + lane];
                        const float sc = ex2f(v.x - Mm);
                        Sm += v.y * sc;
                        Cm += v.z * sc;
                    }
                    const float R0 = (PERSAMPLE ? -Bt * (float)popx : 0.f) - Cc * I2;
                    const float lse2 = R0 + Mm + log2f(Sm + Cm);
                    Ls[i * BM + r] = lse2 * LN2 - logf((float)m_i) -
                                     logf(6.283185307179586f * rho * rho) - log_col_norm;
                }
            }
            if (!ok) break;
            // label normalisation (and the factorised texture posterior) by quarter 0
            if (hf == 0 && live) {
                if (!PERSAMPLE) {
                    float tmax = -INFINITY;
                    for (int i = 0; i < a.n_labels; ++i) {
                        const float rho = a.alpha * fmaxf(sqrtf((float)a.dist2[(size_t)i * P + pq]), a.d_min);
                        int h = 0;
                        for (int w = 0; w < a.Wk; ++w) h += __popc(bx[w & 7] ^ a.rep[i * a.Wk + w]);
                        tmax = fmaxf(tmax, -LOG2E * (float)h / (a.kappa_beta * rho));
                    }
                    float ts = 0.f;
                    for (int i = 0; i < a.n_labels; ++i) {
                        const float rho = a.alpha * fmaxf(sqrtf((float)a.dist2[(size_t)i * P + pq]), a.d_min);
                        int h = 0;
                        for (int w = 0; w < a.Wk; ++w) h += __popc(bx[w & 7] ^ a.rep[i * a.Wk + w]);
                        ts += ex2f(-LOG2E * (float)h / (a.kappa_beta * rho) - tmax);
                    }
                    const float tl = tmax + log2f(ts);
                    for (int i = 0; i < a.n_labels; ++i) {
                        const float rho = a.alpha * fmaxf(sqrtf((float)a.dist2[(size_t)i * P + pq]), a.d_min);
                        int h = 0;
                        for (int w = 0; w < a.Wk; ++w) h += __popc(bx[w & 7] ^ a.rep[i * a.Wk + w]);
                        Ls[i * BM + r] += (-LOG2E * (float)h / (a.kappa_beta * rho) - tl) * LN2;
                    }
                }
                float lmax = -INFINITY;
                for (int i = 0; i < a.n_labels; ++i) lmax = fmaxf(lmax, Ls[i * BM + r]);
                float ls = 0.f;
                for (int i = 0; i < a.n_labels; ++i) ls += expf(Ls[i * BM + r] - lmax);
                const float lse = lmax + logf(ls);
                for (int i = 0; i < a.n_labels; ++i) {
                    const float L = Ls[i * BM + r];
                    a.neglog[(size_t)i * P + pix] = -L;
                    if (a.post) a.post[(size_t)i * P + pix] = expf(L - lse);
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, TMEM_COLS);
    }
}

// Sample tiles laid out exactly as one ring stage: texture slabs (b_j in
// {0, 1}), the colour slab (hi/lo bf16 of I_j and of -C |I_j|^2) and the
// sample coordinates (padded rows: zero operands, far-away coordinates).
template <bool TEX8, int KS, bool PERSAMPLE>
__global__ void build_tiles_kernel(const int32_t* __restrict__ label_off,
                                   const int32_t* __restrict__ tile_off, int n_labels,
                                   int total_tiles, SampleTables t, int n_samples, int k,
                                   float Cc, uint8_t* __restrict__ blob) {
    using C = Cfg<TEX8, KS, PERSAMPLE>;
    const long long gid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (gid >= (long long)total_tiles * BN) return;
    const int tile = (int)(gid / BN), r = (int)(gid % BN);
    int lo = 0, hi = n_labels - 1;  // label of this tile
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tile_off[mid] <= tile) lo = mid; else hi = mid - 1;
    }
    const int i = lo;
    const int s = label_off[i] + (tile - tile_off[i]) * BN + r;
    const bool valid = s < label_off[i + 1];
    uint8_t* st = blob + (size_t)tile * C::stage_bytes;
    if (PERSAMPLE) {
        for (int sl = 0; sl < KS; ++sl) {
            uint32_t wv[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                uint32_t word = 0;
                if (TEX8) {
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int j = 32 * sl + 4 * c + e;
                        if (valid && j < k && ((t.sbits[(size_t)(j >> 5) * n_samples + s] >> (j & 31)) & 1u))
                            word |= 0x38u << (8 * e);
                    }
                } else {
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        const int j = 16 * sl + 2 * c + e;
                        if (valid && j < k && ((t.sbits[(size_t)(j >> 5) * n_samples + s] >> (j & 31)) & 1u))
                            word |= 0x3F80u << (16 * e);
                    }
                }
                wv[c] = word;
            }
            *reinterpret_cast<uint4*>(st + sl * 4096 + tc::slab_off(r, 0)) = make_uint4(wv[0], wv[1], wv[2], wv[3]);
            *reinterpret_cast<uint4*>(st + sl * 4096 + tc::slab_off(r, 16)) = make_uint4(wv[4], wv[5], wv[6], wv[7]);
        }
    }
    uint16_t v[16];
    if (valid) {
        const float R = t.sr[s], G = t.sg[s], B = t.sb[s];
        const float qv = -Cc * fmaf(R, R, fmaf(G, G, B * B));
        uint16_t hr, lr, hg, lg, hb, lb, hq, lq;
        split_bf16(R, hr, lr);
        split_bf16(G, hg, lg);
        split_bf16(B, hb, lb);
        split_bf16(qv, hq, lq);
        const uint16_t vv[16] = {hr, lr, hr, lr, hg, lg, hg, lg, hb, lb, hb, lb, hq, lq, hq, lq};
#pragma unroll
        for (int u = 0; u < 16; ++u) v[u] = vv[u];
    } else {
#pragma unroll
        for (int u = 0; u < 16; ++u) v[u] = 0;
    }
    uint32_t pw[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) pw[c] = v[2 * c] | ((uint32_t)v[2 * c + 1] << 16);
    *reinterpret_cast<uint4*>(st + C::col_off + tc::slab_off(r, 0)) = make_uint4(pw[0], pw[1], pw[2], pw[3]);
    *reinterpret_cast<uint4*>(st + C::col_off + tc::slab_off(r, 16)) = make_uint4(pw[4], pw[5], pw[6], pw[7]);
    reinterpret_cast<float2*>(st + C::xy_off)[r] =
        valid ? make_float2(t.sx[s], t.sy[s]) : make_float2(1.0e15f, 1.0e15f);
}

template <bool TEX8, int KS, bool PERSAMPLE>
cudaError_t run(const TcLaunch& L, cudaStream_t st) {
    using C = Cfg<TEX8, KS, PERSAMPLE>;
    const int total_tiles = L.total_tiles;
    const float Cc = 1.4426950408889634f / (2.f * L.sigma_c2);
    build_tiles_kernel<TEX8, KS, PERSAMPLE><<<(unsigned)(((long long)total_tiles * BN + 127) / 128), 128, 0, st>>>(
        L.d_label_off, L.d_tile_off, L.n_labels, total_tiles, L.t, L.n_samples, L.k, Cc, L.blob);
    TcArgs a{};
    a.img = L.img;
    a.H = L.H;
    a.W = L.W;
    a.bitmask = L.bitmask;
    a.k = L.k;
    a.Wk = (L.k + 31) / 32;
    a.n_labels = L.n_labels;
    a.d_label_off = L.d_label_off;
    a.d_tile_off = L.d_tile_off;
    a.blob = L.blob;
    a.rep = L.t.rep;
    a.dist2 = L.dist2;
    a.alpha = L.alpha;
    a.d_min = L.d_min;
    a.kappa_beta = L.kappa_beta;
    a.sigma_c2 = L.sigma_c2;
    a.neglog = L.neglog;
    a.post = L.post;
    a.d_err = L.d_err;
    const long long P = (long long)L.H * L.W;
    a.n_ptiles = (int)((P + BM - 1) / BM);
    cudaError_t e = cudaFuncSetAttribute(sum_tc_kernel<TEX8, KS, PERSAMPLE>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, C::smem_bytes);
    if (e != cudaSuccess) return e;
    const int grid = a.n_ptiles < L.n_sm ? a.n_ptiles : L.n_sm;
    sum_tc_kernel<TEX8, KS, PERSAMPLE><<<grid, THREADS, C::smem_bytes, st>>>(a);
    return cudaGetLastError();
}

template <bool TEX8, bool PERSAMPLE>
cudaError_t run_ks(const TcLaunch& L, int ks, cudaStream_t st) {
    switch (ks) {
        case 1: return run<TEX8, 1, PERSAMPLE>(L, st);
        case 2: return run<TEX8, 2, PERSAMPLE>(L, st);
        case 3: return run<TEX8, 3, PERSAMPLE>(L, st);
        case 4: return run<TEX8, 4, PERSAMPLE>(L, st);
        case 5: return run<TEX8, 5, PERSAMPLE>(L, st);
        case 6: return run<TEX8, 6, PERSAMPLE>(L, st);
        case 7: return run<TEX8, 7, PERSAMPLE>(L, st);
        case 8: return run<TEX8, 8, PERSAMPLE>(L, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

size_t tc_stage_bytes(int k, bool tex8, bool persample) {
    const int ks = tex8 ? (k + 31) / 32 : (k + 15) / 16;
    return (size_t)(persample ? ks * 4096 : 0) + 4096 + BN * 8;
}

int tc_tiles_per_label(int m) { return (m + BN - 1) / BN; }

bool tc_supported(int k, bool tex8) { return tex8 ? k <= 256 : k <= 128; }

cudaError_t launch_sum_tc(const TcLaunch& L, cudaStream_t st) {
    if (!tc_supported(L.k, L.tex8)) return cudaErrorInvalidValue;
    if (!L.persample) return run_ks<true, false>(L, 1, st);
    const int ks = L.tex8 ? (L.k + 31) / 32 : (L.k + 15) / 16;
    return L.tex8 ? run_ks<true, true>(L, ks, st) : run_ks<false, true>(L, ks, st);
}
