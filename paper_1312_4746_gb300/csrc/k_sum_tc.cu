// Pixel x sample likelihood sum on the tensor cores (tcgen05), the fast form
// of Sec. 3.1 Eq. (color) x Eq. (post_text) (per-sample or factorised).
//
// Per pixel x and label i (log2 units, C = log2(e) / (2 sigma_c2),
// Bt = log2(e) / beta_i(x), nA = -log2(e) / (2 rho_i(x)^2), f = nA / Bt):
//   e_j = nA |x - x_j|^2 - C |I - I_j|^2 - Bt TSM(b_x, b_j)
//       = Bt D1_j + nA |x'|^2 + R0,
//   D1_j = sum_t (2 b_x,t - 1) b_j,t  +  (1/Bt) (2 C I.I_j - C |I_j|^2)
//          + f (-2 x'.u_j + |u_j|^2),                R0 = -Bt |b_x| - C |I|^2,
// where x' = x - o and u_j = x_j - o relative to the centre o of the pixel
// tile, so that |x - x_j|^2 = |x'|^2 - 2 x'.u_j + |u_j|^2 with |x'| <= 9:
// the location terms carry the magnitude of |x - x_j|^2 itself (no
// cancellation between large offsets). One FP32 accumulator per sample
// receives all of it from tcgen05 MMAs: the texture sum (an exact integer,
// 2 b_x.b_j - |b_j|, so TSM = |b_x| minus it) from FP8 (e4m3, values 0 and
// +-1) or BF16 MMAs over whole 32-code (16-code) slabs, the last few codes
// (k mod 32 or k mod 16, when at most EXT_MAX) riding in the second half of
// the second location slab as BF16 +-1 / 0; the colour part from a 16-wide
// BF16 MMA over hi/lo splits of both factors (relative error about 2^-17);
// the location part from two 16-wide BF16 MMAs whose sample side is exact
// (2u in two bf16 pieces per axis, |u|^2 in four) and whose pixel side
// holds three-piece splits of -f x' and f (relative error below 2^-24). The
// sample side of the location is formed per (pixel tile, sample tile) by the
// producer from the sample positions (the rest of the sample side is laid
// out once per call and bulk-copied); the pixel side per label by the
// epilogue. In the factorised form D1 holds the colour and location parts
// with Bt = 1.
//
// All full exponents are <= 0, so no running maximum is needed: the row sum
// accumulates 2^(e + shift) with a fixed shift 96 - ceil(log2 m_i) (no term
// above 2^96 / m_i, no overflow), in packed f32x2 arithmetic, TwoSum-
// compensated across 16-sample chunks. A label row goes to the FP64
// recompute (refine_fp64_kernel) when it totals less than m_i 2^-100 (terms
// may have underflowed) or when its a-priori error bound exceeds
// l_tol max(|L|, 1) (derivation at the flagging site).
//
// Work items are (image, 16 x 8 pixel tile, label): all sample tiles of one
// label for one pixel tile (one TMEM lane per pixel, one TMEM column per
// sample of a 128-sample tile), numbered image by image, pixel tile by pixel
// tile, label by label. The persistent CTAs claim work from global counters:
// whole pixel tiles (all their labels, consecutive items) until about one
// pixel tile per CTA is left, then single items, each CTA one claim ahead of
// its producers, so that the two CTAs sharing an SM, which do not run at the
// same speed, and all SMs finish within about one item of each other. A CTA
// passes its claims (runs of consecutive items) to its roles through a small
// ring in shared memory. The label normalisation runs in a separate pass
// once every label row is written.
//
// Two persistent CTAs per SM (one where the shared-memory layout does not
// fit twice).
//   warps 8..11  producers: per stage, one bulk-copies (TMA) the
//                pre-laid-out part of a sample tile (texture slabs, colour
//                slab, the texture codes beyond the texture slabs), and all
//                four write its location rows for this pixel tile (32
//                samples each)
//   warp 12      MMA issuer: D1 <- texture slabs + colour slab + location
//                slabs; TMEM double-buffered (2 x 128 columns per CTA), so
//                one tile's MMAs run while the epilogue reads the previous
//   warps 0..7   epilogue: writes the pixel-side colour and location rows
//                of the NEXT item while it sums the current one (two label
//                buffers), so that the MMAs run on across label boundaries;
//                warp w reads lanes 32 (w % 4) .. +31 and columns
//                64 (w / 4) .. +63 of each tile (16-column loads), merges the
//                two column parts per item (16 warps of 32 columns in the
//                one-CTA layout).
// Every mbarrier wait is bounded by the global timer; on expiry the CTA sets
// the device error word, stops issuing, drains its copies and MMAs, frees its
// tensor memory and exits.
#include <cuda_bf16.h>

#include <cstdint>
#include <type_traits>

#include "internal.h"
#include "tc_ptx.cuh"

namespace {

constexpr int BM = 128, BN = 128;
constexpr int TW = 16, TH = 8;          // pixel tile 16 x 8
constexpr float LOG2E = 1.4426950408889634f;
constexpr float LN2 = 0.6931471805599453f;
constexpr uint64_t WAIT_NS = 1000000000ull;  // 1 s per wait
constexpr uint32_t SUSPEND_NS = 1000u;       // longest suspension of one barrier test
// The sum runs on 2^(e + SHIFT_i) with SHIFT_i = 96 - ceil(log2 m_i): every
// term is <= 2^96 / m_i, so the row sum stays below 2^96. A shifted total
// below m_i 2^-100 may have lost mass to FP32 underflow (each lost term is
// < 2^-126, at most m_i of them: relative loss < 2^-26) and is recomputed.
constexpr float FLOOR_PER_SAMPLE = 7.888609052210118e-31f;  // 2^-100

struct TcArgs {
    const TcImage* images;  // n_images descriptors, in launch (first_item) order
    int n_images;
    long long n_items;      // items over all images
    long long total_pixels; // pixels over all images
    int pt1;                // pixel tiles claimed whole, with all their labels
    long long i1;           // first item claimed on its own (the rest, after them)
    int k, Wk;
    int ext;                // texture codes carried in the second location slab
    float alpha, d_min, kappa_beta, sigma_c2;
    bool rho_var;   // rho is the location kernel's variance (else its standard deviation)
    int* d_err;
    int4* fb_list;  // (image, pixel) of pixels with flagged label rows
    int* fb_count;
    int fb_cap;
    unsigned* queue;           // claim counters: whole pixel tiles, single items
    unsigned long long* flags; // per pixel: label rows flagged for the FP64 recompute
    float l_tol;    // relative tolerance on L of the a-priori row bound (0: off)
    uint64_t wait_ns;  // time limit of each barrier wait (0: WAIT_NS)
    bool stall;        // the MMA issuer of the last CTA waits on a barrier nobody completes
};

// A work item: image, pixel tile, label (img == -1: no more items).
struct Item {
    int img, pt, lab;
};

// Item number n (0 <= n < n_items), or none.
__device__ Item item_of(const TcArgs& a, long long n) {
    Item it{-1, 0, 0};
    if (n < 0 || n >= a.n_items) return it;
    int lo = 0, hi = a.n_images - 1;  // the last image whose first item is <= n
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.images[mid].first_item <= n) lo = mid; else hi = mid - 1;
    }
    const TcImage& m = a.images[lo];
    const long long local = n - m.first_item;
    it.img = lo;
    it.pt = (int)(local / m.n_labels);
    it.lab = (int)(local - (long long)it.pt * m.n_labels);
    return it;
}

// Image of pixel tile number t of the launch (the last image whose first
// pixel tile is <= t).
__device__ __forceinline__ int ptile_image(const TcArgs& a, int t) {
    int lo = 0, hi = a.n_images - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.images[mid].first_ptile <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Ring of claims in shared memory: entry e (a run of consecutive item
// numbers: first, count; count 0 marks the end) sits in slot e % QD;
// q_full[slot] completes when it is written, q_empty[slot] when every reader
// has taken it. Depth QD covers the claimer's lead over the slowest reader
// (one claim of look-ahead, the producers' sample tiles in flight and the
// epilogue's one item of look-ahead, each item at least one tile).
constexpr int QD = 16;

// A reader's place in the ring: the entry it holds and the item within it.
struct RingPos {
    int e = -1, first = 0, count = 0, k = 0;
};

// Texture codes in the MMA slabs and in the second location slab: whole
// slabs of 32 (FP8) or 16 (BF16) codes, and the remaining k mod 32 (16)
// codes in the second half of the second location slab (EXT_MAX columns)
// when they fit there, else one more slab.
constexpr int EXT_MAX = 8;
__host__ __device__ constexpr int tex_slabs(int k, bool tex8) {
    return tex8 ? (k % 32 <= EXT_MAX ? k / 32 : k / 32 + 1)
                : (k % 16 <= EXT_MAX ? k / 16 : k / 16 + 1);
}
__host__ __device__ constexpr int tex_ext(int k, bool tex8) {
    return k - tex_slabs(k, tex8) * (tex8 ? 32 : 16) > 0 ? k - tex_slabs(k, tex8) * (tex8 ? 32 : 16)
                                                           : 0;
}

template <bool TEX8, int KS, bool PERSAMPLE, bool SOLO = false>
struct Cfg {
    // ring stage: the second location slab L1 in halves (tc::halves_off;
    // the first half, location pieces, written by the producer; the second,
    // the texture codes beyond the texture slabs, bulk-copied), the texture
    // slabs and the colour slab (bulk-copied with L1's second half), then
    // the first location slab L0 (producer)
    static constexpr int tex_bytes = PERSAMPLE ? KS * 4096 : 0;
    static constexpr int l1_off = 0;
    static constexpr int copy_off = 2048;                     // bulk-copied part of a stage
    static constexpr int tex_off = 4096;
    static constexpr int col_off = 4096 + tex_bytes;
    static constexpr int copy_bytes = 2048 + tex_bytes + 4096;
    static constexpr int l0_off = 8192 + tex_bytes;
    static constexpr int stage_bytes = tex_bytes + 3 * 4096;
    static constexpr int NB = 2;                              // D1 accumulators (128 columns each)
    static constexpr uint32_t TMEM_COLS = 128u * NB;
    static constexpr int XB = 2 * NB;                         // item-merge exchange buffers
    static constexpr int AP = 3 * 4096;                       // pixel-side colour + L0 + L1 slabs
    // Two CTAs per SM (each 256 TMEM columns, a sample ring of two or more
    // stages, 8 epilogue warps) when that layout fits twice in the SM's
    // 228 KB (a CTA of the pair may use 228 KB / 2 - 1 KB, the per-CTA
    // reservation) and SOLO is not asked for, else one CTA per SM with 16
    // epilogue warps and the deeper ring that the whole SM's shared memory
    // allows. The shapes split a sample tile's columns differently among the
    // epilogue warps, so their compensated sums associate differently: the
    // results agree to rounding, within the same a-priori bound. Two label
    // buffers of pixel-side operands always (the next item's are written
    // while the current one is summed); the sample ring as deep as fits (2 to
    // 4 stages) and, if room is left, two pixel-tile texture buffers.
    static constexpr int PAIR_LIMIT = 228 * 1024 / 2 - 1024;
    static constexpr int MISC = 16 + 8 * QD;  // TMEM base, abort flag, claim ring
    static constexpr int bytes(int stages, int atb, int epq) {
        return stages * stage_bytes + atb * tex_bytes + 2 * AP + XB * (epq - 1) * 4 * 32 * 8 +
               (2 * stages + 2 * NB + 4 + 2 * atb + 4 * XB + 1 + 2 * QD) * 8 + MISC;
    }
    static constexpr bool PAIR = !SOLO && bytes(2, 1, 2) <= PAIR_LIMIT;
    static constexpr int MIN_BLOCKS = PAIR ? 2 : 1;
    static constexpr int EPQ = PAIR ? 2 : 4;                 // epilogue warps per TMEM lane quadrant
    static constexpr int EPI_WARPS = 4 * EPQ;
    static constexpr int CPW = BN / EPQ;                     // columns per epilogue warp per tile
    static constexpr int NPROD = 4;                          // producer warps
    static constexpr int PRODUCER = EPI_WARPS;
    static constexpr int MMA_WARP = EPI_WARPS + NPROD;
    static constexpr int THREADS = (EPI_WARPS + NPROD + 1) * 32;
    static constexpr int LIMIT = PAIR ? PAIR_LIMIT : 227 * 1024;
    // two pixel-tile texture buffers whenever they fit with a two-stage ring
    // (claimed items seldom share a pixel tile), then the ring as deep as fits
    static constexpr int ATB = bytes(2, 2, EPQ) <= LIMIT ? 2 : 1;
    static constexpr int STAGES = bytes(4, ATB, EPQ) <= LIMIT ? 4 : bytes(3, ATB, EPQ) <= LIMIT ? 3 : 2;
    // shared memory map
    static constexpr int ring_off = 0;
    static constexpr int atex_off = ring_off + STAGES * stage_bytes;
    static constexpr int acol_off = atex_off + ATB * tex_bytes;
    static constexpr int xchg_off = acol_off + 2 * AP;               // [XB][EPQ-1][4][32] float2
    static constexpr int bar_off = xchg_off + XB * (EPQ - 1) * 4 * 32 * 8;
    static constexpr int n_bars = 2 * STAGES + 2 * NB + 4 + 2 * ATB + 4 * XB + 1 + 2 * QD;
    static constexpr int misc_off = bar_off + n_bars * 8;
    // a floor on the shared memory keeps a third CTA (or, unpaired, a
    // second) off the SM, so that tensor memory allocation never waits
    static constexpr int smem_floor = PAIR ? 80 * 1024 : 120 * 1024;
    static constexpr int smem_bytes = misc_off + MISC > smem_floor ? misc_off + MISC : smem_floor;
    static_assert(misc_off + MISC == bytes(STAGES, ATB, EPQ), "layout size");
    static_assert(bytes(STAGES, ATB, EPQ) <= LIMIT, "shared-memory layout");
    static constexpr uint32_t id_tex = TEX8 ? tc::idesc(BM, BN, 0, 0) : tc::idesc(BM, BN, 1, 1);
    static constexpr uint32_t id_bf16 = tc::idesc(BM, BN, 1, 1);
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
__device__ __forceinline__ uint32_t pack2(uint16_t a, uint16_t b) { return a | ((uint32_t)b << 16); }

__device__ __forceinline__ void set_abort(volatile int* abort_flag, int* d_err, int site) {
    *abort_flag = 1;
    if (atomicCAS(d_err, 0, CS_DEVERR_TIMEOUT) == 0) d_err[1] = site;
}

// Single-thread bounded wait. Each test may suspend the thread for up to
// 1 us (it resumes when the phase completes), so a waiting warp takes no
// issue slots from the working warps of the SM's other CTA; the timer is
// read every 256 tests.
__device__ __forceinline__ bool spin_bar(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                         int* d_err, int site, uint64_t wait_ns) {
    if (*abort_flag) return false;
    uint64_t deadline = 0;
    for (uint32_t n = 0;; ++n) {
        if (tc::mbar_try_wait(bar, parity, SUSPEND_NS)) return true;
        if ((n & 255u) == 255u) {
            const uint64_t now = tc::globaltimer();
            if (deadline == 0) deadline = now + wait_ns;
            else if (now > deadline) break;
        }
    }
    set_abort(abort_flag, d_err, site);
    return false;
}

// Warp-uniform bounded wait (every lane tests the same phase, so the warp
// stays converged); suspending tests as in spin_bar.
__device__ __forceinline__ bool spin_warp(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                          int* d_err, int site, uint64_t wait_ns) {
    uint64_t deadline = 0;
    for (uint32_t n = 0;; ++n) {
        if (__all_sync(0xffffffffu, tc::mbar_try_wait(bar, parity, SUSPEND_NS))) return true;
        if ((n & 255u) == 255u) {
            int late = 0;
            if ((threadIdx.x & 31) == 0) {
                const uint64_t now = tc::globaltimer();
                if (deadline == 0) deadline = now + wait_ns;
                else late = now > deadline || *abort_flag;
            }
            if (__shfl_sync(0xffffffffu, late, 0)) break;
        }
    }
    if ((threadIdx.x & 31) == 0) set_abort(abort_flag, d_err, site);
    return false;
}

__device__ __forceinline__ int tiles_of(const int32_t* tile_off, int i) {
    return tile_off[i + 1] - tile_off[i];
}

// Sample-side location rows (a 16-wide slab L0 and the first half of L1)
// of a sample at packed position w (x | y << 16) relative to the pixel
// tile's centre (cx, cy), u = x_j - centre: 2u per axis in two exact bf16
// pieces (h, l), |u|^2 (< 2^31) in four exact bf16 pieces q0..q3:
//   L0 = [hx lx hx lx hx lx  hy ly hy ly hy ly  q0 q1 q2 q3],
//   L1 = [q0 q1 q2 q0 q1  0 0 0 | b0 .. b7],
// where the second half of L1, the sample's texture codes beyond the
// texture slabs (code 32 KS + e, or 16 KS + e) as bf16 1 / 0, does not depend
// on the pixel tile and is laid out with the sample tile (build_tiles_kernel);
// the pixel side holds the matching pieces of -f x' and f (see the
// epilogue) and +-1 for the texture codes. The pieces are bit fields of the
// integers (at most 8 significant bits each, so exact in bf16):
// 2u = (2u & ~255) + (2u & 255) and |u|^2 by bytes from its leading bit
// down. A padded sample has q0 = 2^30 and zeros elsewhere, so that its
// exponent vanishes.
__device__ __forceinline__ uint32_t bf16_exact(int v) {  // v has <= 8 significant bits
    return __float_as_uint((float)v) >> 16;
}
__device__ __forceinline__ void loc_row_b(uint32_t w, int cx, int cy, bool valid, uint4& l0a,
                                          uint4& l0b, uint4& l1a) {
    if (!valid) {
        l0a = make_uint4(0, 0, 0, 0);
        l0b = make_uint4(0, 0, bf16_exact(1 << 30), 0);
        l1a = make_uint4(0, 0, 0, 0);
        return;
    }
    const int ux = (int)(w & 0xFFFFu) - cx, uy = (int)(w >> 16) - cy;  // |u| < 2^15
    const int vx = 2 * ux, vy = 2 * uy;
    const uint32_t px = bf16_exact(vx & ~255) | (bf16_exact(vx & 255) << 16);
    const uint32_t py = bf16_exact(vy & ~255) | (bf16_exact(vy & 255) << 16);
    // |u|^2 in bytes below its leading bit: q0 = bits [k, k + 8), q1 = bits
    // [k - 8, k), ... (k = max(lead - 7, 0)), so that each piece is at most
    // 2^-8 of the one before and the pixel side may drop the smallest products
    const uint32_t q = (uint32_t)(ux * ux + uy * uy);
    const int k0 = max(24 - __clz((int)q), 0), k1 = max(k0 - 8, 0), k2 = max(k0 - 16, 0);
    const uint32_t q0 = bf16_exact((int)(q & (0xFFu << k0))),
                   q1 = bf16_exact((int)(q & (0xFFu << k1) & ((1u << k0) - 1u))),
                   q2 = bf16_exact((int)(q & (0xFFu << k2) & ((1u << k1) - 1u))),
                   q3 = bf16_exact((int)(q & ((1u << k2) - 1u)));
    l0a = make_uint4(px, px, px, py);
    l0b = make_uint4(py, py, q0 | (q1 << 16), q2 | (q3 << 16));
    l1a = make_uint4(q0 | (q1 << 16), q2 | (q0 << 16), q1, 0u);
}

// Three bf16 pieces of an FP32 value (each the rounding of the exact
// remainder; v = p1 + p2 + p3 + r with |r| <= 2^-24 |v|).
__device__ __forceinline__ void split3_bf16(float v, uint16_t& p1, uint16_t& p2, uint16_t& p3) {
    const __nv_bfloat16 b1 = __float2bfloat16_rn(v);
    const float r1 = v - __bfloat162float(b1);
    const __nv_bfloat16 b2 = __float2bfloat16_rn(r1);
    const float r2 = r1 - __bfloat162float(b2);
    p1 = __bfloat16_as_ushort(b1);
    p2 = __bfloat16_as_ushort(b2);
    p3 = bf16_bits(r2);
}

// Packed FP32 pairs (Blackwell f32x2 instructions: one issue, two lanes of
// work) on 64-bit registers holding (low, high) = (element 0, element 1).
__device__ __forceinline__ uint64_t pk2(float lo, float hi) {
    uint64_t d;
    asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(lo), "f"(hi));
    return d;
}
__device__ __forceinline__ uint64_t fma2(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ uint64_t add2(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
// 2^x of both halves.
__device__ __forceinline__ uint64_t ex2x2(uint64_t v) {
    uint64_t d;
    asm("{\n\t.reg .f32 x, y;\n\tmov.b64 {x, y}, %1;\n\t"
        "ex2.approx.ftz.f32 x, x;\n\tex2.approx.ftz.f32 y, y;\n\t"
        "mov.b64 %0, {x, y};\n\t}"
        : "=l"(d)
        : "l"(v));
    return d;
}
__device__ __forceinline__ float lo32(uint64_t v) { return __uint_as_float((uint32_t)v); }
__device__ __forceinline__ float hi32(uint64_t v) { return __uint_as_float((uint32_t)(v >> 32)); }

// Sum over 16 columns of one pixel row of 2^e, e = Bt D1 + k (log2 units,
// shifted full exponents); r1 holds D1 as packed column pairs. Full chunk:
// packed arithmetic; partial chunk: the first nv.
__device__ __forceinline__ float sum16_full(const uint64_t (&r1)[8], uint64_t bt2, uint64_t k2) {
    uint64_t acc0 = 0, acc1 = 0;  // (0.f, 0.f)
#pragma unroll
    for (int u = 0; u < 8; u += 2) {
        acc0 = add2(acc0, ex2x2(fma2(bt2, r1[u], k2)));
        acc1 = add2(acc1, ex2x2(fma2(bt2, r1[u + 1], k2)));
    }
    const uint64_t t = add2(acc0, acc1);
    return lo32(t) + hi32(t);
}
__device__ __forceinline__ float sum16_part(const uint64_t (&r1)[8], int nv, uint64_t bt2,
                                            uint64_t k2) {
    float t0 = 0.f, t1 = 0.f;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        const uint64_t v = fma2(bt2, r1[u], k2);
        t0 += 2 * u < nv ? ex2f(lo32(v)) : 0.f;
        t1 += 2 * u + 1 < nv ? ex2f(hi32(v)) : 0.f;
    }
    return t0 + t1;
}
// (S, Cc) += ts by TwoSum.
__device__ __forceinline__ void two_sum(float ts, float& S, float& Cc) {
    const float sn = S + ts;
    const float bb = sn - S;
    Cc += (S - (sn - bb)) + (ts - bb);
    S = sn;
}

// Label normalisation of one pixel once every label row is in the output
// plane: the factorised form's majority-co-support texture posterior is added
// first, then the posteriors softmax_i L_i.
template <bool PERSAMPLE>
__device__ void normalise_pixel(const TcArgs& a, const TcImage& im, int pix, const uint32_t* bxp) {
    const long long P = (long long)im.H * im.W;
    float* nl = im.neglog + pix;
    if (!PERSAMPLE && im.rep) {  // factorised: the majority-co-support posterior
        float tmax = -INFINITY;
        for (int i = 0; i < im.n_labels; ++i) {
            const float rho = a.alpha * fmaxf(sqrtf((float)im.dist2[(size_t)i * P + pix]), a.d_min);
            int h = 0;
            for (int w = 0; w < a.Wk; ++w) h += __popc(bxp[w] ^ im.rep[i * a.Wk + w]);
            tmax = fmaxf(tmax, -LOG2E * (float)h / (a.kappa_beta * rho));
        }
        float ts = 0.f;
        for (int i = 0; i < im.n_labels; ++i) {
            const float rho = a.alpha * fmaxf(sqrtf((float)im.dist2[(size_t)i * P + pix]), a.d_min);
            int h = 0;
            for (int w = 0; w < a.Wk; ++w) h += __popc(bxp[w] ^ im.rep[i * a.Wk + w]);
            ts += ex2f(-LOG2E * (float)h / (a.kappa_beta * rho) - tmax);
        }
        const float tl = tmax + log2f(ts);
        for (int i = 0; i < im.n_labels; ++i) {
            const float rho = a.alpha * fmaxf(sqrtf((float)im.dist2[(size_t)i * P + pix]), a.d_min);
            int h = 0;
            for (int w = 0; w < a.Wk; ++w) h += __popc(bxp[w] ^ im.rep[i * a.Wk + w]);
            nl[(size_t)i * P] = nl[(size_t)i * P] -
                                (-LOG2E * (float)h / (a.kappa_beta * rho) - tl) * LN2;
        }
    }
    float lmax = -INFINITY;
    for (int i = 0; i < im.n_labels; ++i) lmax = fmaxf(lmax, -nl[(size_t)i * P]);
    float ls = 0.f;
    for (int i = 0; i < im.n_labels; ++i) ls += expf(-nl[(size_t)i * P] - lmax);
    const float lse = lmax + logf(ls);
    if (im.post)
        for (int i = 0; i < im.n_labels; ++i)
            im.post[(size_t)i * P + pix] = expf(-nl[(size_t)i * P] - lse);
}

// The normalisation pass after the sum: one thread per pixel of every image
// of the launch; pixels with a flagged label row are left to the FP64
// recompute, which normalises them in double.
template <bool PERSAMPLE>
__global__ void __launch_bounds__(256) normalise_kernel(TcArgs a) {
    for (long long gp = blockIdx.x * 256ll + threadIdx.x; gp < a.total_pixels;
         gp += (long long)gridDim.x * 256) {
        int lo = 0, hi = a.n_images - 1;  // the last image whose first pixel is <= gp
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (a.images[mid].pix_off <= gp) lo = mid; else hi = mid - 1;
        }
        const TcImage& im = a.images[lo];
        const int pix = (int)(gp - im.pix_off);
        if (a.flags[gp] != 0ull) continue;
        normalise_pixel<PERSAMPLE>(a, im, pix, im.bitmask + (size_t)pix * a.Wk);
    }
}

template <bool TEX8, int KS, bool PERSAMPLE, bool SOLO>
__global__ void __launch_bounds__((Cfg<TEX8, KS, PERSAMPLE, SOLO>::THREADS),
                                  (Cfg<TEX8, KS, PERSAMPLE, SOLO>::MIN_BLOCKS)) sum_tc_kernel(TcArgs a) {
    using C = Cfg<TEX8, KS, PERSAMPLE, SOLO>;
    constexpr int EPQ = C::EPQ, EPI_WARPS = C::EPI_WARPS, CPW = C::CPW, NB = C::NB, ATB = C::ATB;
    constexpr int PRODUCER = C::PRODUCER, MMA_WARP = C::MMA_WARP;
    // With as many ring stages as accumulators, stage it % STAGES and
    // accumulator it % NB free up with the same MMAs: the producers then wait
    // on the accumulator's commit and the MMA issuer commits once per tile.
    constexpr bool ONE_COMMIT = C::STAGES == NB;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t* ring = smem + C::ring_off;
    uint8_t* atex = smem + C::atex_off;
    uint8_t* acol = smem + C::acol_off;
    float2* xchg = reinterpret_cast<float2*>(smem + C::xchg_off);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + C::bar_off);
    uint64_t* full = bars;                        // [STAGES] producer arrivals + TMA bytes
    uint64_t* empty = full + C::STAGES;           // [STAGES] MMA commit
    uint64_t* tmem_full = empty + C::STAGES;      // [NB] MMA commit
    uint64_t* tmem_empty = tmem_full + NB;        // [NB] epilogue warps
    uint64_t* acol_full = tmem_empty + NB;        // [2] epilogue warps
    uint64_t* acol_empty = acol_full + 2;         // [2] MMA commit
    uint64_t* atex_full = acol_empty + 2;         // [ATB] epilogue warps
    uint64_t* atex_empty = atex_full + ATB;       // [ATB] MMA commit
    uint64_t* xchg_full = atex_empty + ATB;       // [XB buffers][4 quadrants]
    uint64_t* stall_bar = xchg_full + 4 * C::XB;  // [1] nobody arrives (timeout-path tests)
    uint64_t* q_full = stall_bar + 1;             // [QD] item ring: entry written
    uint64_t* q_empty = q_full + QD;              // [QD] item ring: entry read by every reader
    uint32_t* tmem_base_s = reinterpret_cast<uint32_t*>(smem + C::misc_off);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + C::misc_off + 4);
    int* qfirst = reinterpret_cast<int*>(smem + C::misc_off + 16);  // [QD] first item of a claim
    int* qcount = qfirst + QD;                                      // [QD] its items, 0: end

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint64_t wait_ns = a.wait_ns ? a.wait_ns : WAIT_NS;

    if (threadIdx.x == 0) {
        for (int s = 0; s < C::STAGES; ++s) {
            tc::mbar_init(full + s, C::NPROD);
            tc::mbar_init(empty + s, 1);
        }
        for (int b = 0; b < NB; ++b) {
            tc::mbar_init(tmem_full + b, 1);
            tc::mbar_init(tmem_empty + b, EPI_WARPS);
        }
        for (int b = 0; b < 2; ++b) {
            tc::mbar_init(acol_full + b, EPI_WARPS);
            tc::mbar_init(acol_empty + b, 1);
        }
        for (int b = 0; b < ATB; ++b) {
            tc::mbar_init(atex_full + b, EPI_WARPS);
            tc::mbar_init(atex_empty + b, 1);
        }
        for (int x = 0; x < 4 * C::XB; ++x) tc::mbar_init(xchg_full + x, EPQ - 1);
        tc::mbar_init(stall_bar, 1);
        for (int x = 0; x < QD; ++x) {
            tc::mbar_init(q_full + x, 1);
            // readers: the producer warps, the MMA issuer, the epilogue warps
            tc::mbar_init(q_empty + x, C::NPROD + 1 + EPI_WARPS);
        }
        *abort_flag = 0;
        tc::fence_mbar_init();
    }
    if (warp == 0) {
        tc::tmem_alloc(tmem_base_s, C::TMEM_COLS);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_base_s;
    // the next item number of a reader (-1: no more items), from its current
    // claim or the next ring entry; `single`: one thread reads (the MMA
    // issuer), else a whole warp (lane 0 releases the slot)
    auto next_num = [&](RingPos& r, int& num, bool single) {
        if (r.e >= 0 && r.k + 1 < r.count) {
            num = r.first + ++r.k;
            return true;
        }
        ++r.e;
        const int slot = r.e % QD;
        const uint32_t par = (uint32_t)((r.e / QD) & 1);
        if (!(single ? spin_bar(q_full + slot, par, abort_flag, a.d_err, 14, wait_ns)
                     : spin_warp(q_full + slot, par, abort_flag, a.d_err, 13, wait_ns)))
            return false;
        r.first = qfirst[slot];
        r.count = qcount[slot];
        r.k = 0;
        if (!single) __syncwarp();
        if (single || (threadIdx.x & 31) == 0) tc::mbar_arrive(q_empty + slot);
        num = r.count > 0 ? r.first : -1;
        return true;
    };

    if (warp >= PRODUCER && warp < PRODUCER + C::NPROD) {
        const int pw = warp - PRODUCER;  // producer warp: rows 32 u + lane, u = pw mod NPROD
        // ------------------------------------------------------------ producer
        uint32_t it = 0;  // tiles issued by this CTA (< 2^32 in any launch)
        bool ok = true;
        constexpr int RV = BN / 32 / C::NPROD;  // rows of 32 samples per producer warp
        int nclaimed = 0;           // warp 0: ring entries written
        bool claims_ended = false;  // warp 0: the end marker is written
        bool single = false;        // warp 0: the whole pixel tiles are gone
        RingPos rp;
        while (ok) {
            // warp 0 keeps the ring one claim ahead of its own reads: the
            // claim after the one it is about to start (the epilogue prepares
            // each next item's operands while it sums the current one)
            if (pw == 0) {
                while (!claims_ended && nclaimed <= rp.e + 2) {
                    const int slot = nclaimed % QD;
                    ok = spin_warp(q_empty + slot, (uint32_t)(((nclaimed / QD) & 1) ^ 1), abort_flag,
                                   a.d_err, 12, wait_ns);
                    if (!ok) break;
                    int cnt = 0;
                    if (lane == 0) {
                        int first = 0;
                        if (!single) {
                            const unsigned t = atomicAdd(a.queue, 1u);
                            if ((long long)t < a.pt1) {
                                const int g = ptile_image(a, (int)t);
                                const TcImage& m = a.images[g];
                                first = (int)(m.first_item + (long long)(t - m.first_ptile) * m.n_labels);
                                cnt = m.n_labels;
                            } else {
                                single = true;
                            }
                        }
                        if (single) {
                            const long long i = a.i1 + atomicAdd(a.queue + 1, 1u);
                            first = (int)i;
                            cnt = i < a.n_items ? 1 : 0;
                        }
                        qfirst[slot] = first;
                        qcount[slot] = cnt;
                        tc::mbar_arrive(q_full + slot);  // releases the entry to the readers
                    }
                    cnt = __shfl_sync(0xffffffffu, cnt, 0);
                    single = __shfl_sync(0xffffffffu, (int)single, 0) != 0;
                    claims_ended = cnt == 0;
                    ++nclaimed;
                }
                if (!ok) break;
            }
            int num = -1;
            ok = next_num(rp, num, false);
            if (!ok || num < 0) break;
            const Item itm = item_of(a, num);
            const TcImage& im = a.images[itm.img];
            // centre of the pixel tile: the origin of the location operands
            const int cx = (itm.pt % im.ntx) * TW + TW / 2, cy = (itm.pt / im.ntx) * TH + TH / 2;
            const int T0 = im.tile_off[itm.lab], T1 = im.tile_off[itm.lab + 1];
            const int m_i = im.label_off[itm.lab + 1] - im.label_off[itm.lab];
            // sample positions one tile ahead
            uint32_t w_next[RV];
#pragma unroll
            for (int v = 0; v < RV; ++v)
                w_next[v] = im.tile_xy[(size_t)T0 * BN + 32 * (pw + C::NPROD * v) + lane];
            for (int T = T0; ok && T < T1; ++T, ++it) {
                uint32_t w[RV];
#pragma unroll
                for (int v = 0; v < RV; ++v) {
                    w[v] = w_next[v];
                    if (T + 1 < T1)
                        w_next[v] = im.tile_xy[(size_t)(T + 1) * BN + 32 * (pw + C::NPROD * v) + lane];
                }
                const int s = (int)(it % C::STAGES);
                const uint32_t ph = (uint32_t)((it / C::STAGES) & 1);
                ok = spin_warp((ONE_COMMIT ? tmem_full : empty) + s, ph ^ 1, abort_flag, a.d_err, 1,
                               wait_ns);
                if (!ok) break;
                uint8_t* st = ring + s * C::stage_bytes;
                const int nvalid = min(BN, m_i - (T - T0) * BN);
                // the copy first, so that it lands while the location rows
                // are written; the arrival follows them
                if (pw == 0 && lane == 0) {
                    tc::mbar_expect_tx(full + s, C::copy_bytes);
                    tc::bulk_g2s(st + C::copy_off, im.blob + (size_t)T * C::copy_bytes, C::copy_bytes,
                                 full + s);
                }
#pragma unroll
                for (int v = 0; v < RV; ++v) {
                    const int j = 32 * (pw + C::NPROD * v) + lane;
                    uint4 l0a, l0b, l1a;
                    loc_row_b(w[v], cx, cy, j < nvalid, l0a, l0b, l1a);
                    *reinterpret_cast<uint4*>(st + C::l0_off + tc::slab_off(j, 0)) = l0a;
                    *reinterpret_cast<uint4*>(st + C::l0_off + tc::slab_off(j, 16)) = l0b;
                    *reinterpret_cast<uint4*>(st + C::l1_off + tc::halves_off(j, 0)) = l1a;
                }
                tc::fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(full + s);
            }
        }
        // drain: copies still in flight must land before the CTA exits
        if (pw == 0 && lane == 0)
            for (uint32_t d = (it > C::STAGES ? it - C::STAGES : 0); d < it; ++d)
                tc::mbar_wait(full + (int)(d % C::STAGES), (uint32_t)((d / C::STAGES) & 1),
                              tc::globaltimer() + wait_ns);
    } else if (warp == MMA_WARP) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            uint32_t it = 0, li = 0, ptc = 0;  // tiles, items, pixel tiles started
            bool ok = true;
            long long last = -1;
            // test hook: nothing has been issued yet, so every other role
            // drains cleanly once this wait gives up and raises the abort flag
            if (a.stall && blockIdx.x == gridDim.x - 1)
                ok = spin_bar(stall_bar, 0, abort_flag, a.d_err, 2, wait_ns);
            RingPos rp;  // the MMA issuer is lane 0 alone: it reads the ring itself
            int num = -1;
            ok = ok && next_num(rp, num, true);
            Item itm = item_of(a, num);
            int cur_img = -1, cur_pt = -1;
            while (ok && itm.img >= 0) {
                const TcImage& im = a.images[itm.img];
                if (itm.img != cur_img || itm.pt != cur_pt) {  // a new pixel tile
                    ok = spin_bar(atex_full + (int)(ptc % ATB), (uint32_t)((ptc / ATB) & 1),
                                  abort_flag, a.d_err, 3, wait_ns);
                    cur_img = itm.img;
                    cur_pt = itm.pt;
                    ++ptc;
                }
                const int cb = (int)(li & 1);
                ok = ok && spin_bar(acol_full + cb, (uint32_t)((li >> 1) & 1), abort_flag, a.d_err,
                                    4, wait_ns);
                // descriptor low words: colour, L0, L1 slabs of this item and
                // this pixel tile's texture slabs (tc::desc_lo)
                const uint32_t ap = tc::desc_lo(acol + cb * C::AP);
                const uint32_t ax = tc::desc_lo(atex + (int)((ptc - 1) % ATB) * C::tex_bytes);
                const uint32_t ring_lo = tc::desc_lo(ring);
                const int nt = tiles_of(im.tile_off, itm.lab);
                for (int t = 0; ok && t < nt; ++t, ++it) {
                    const int s = (int)(it % C::STAGES), b = (int)(it % NB);
                    ok = spin_bar(full + s, (uint32_t)((it / C::STAGES) & 1), abort_flag, a.d_err, 5,
                                  wait_ns) &&
                         spin_bar(tmem_empty + b, (uint32_t)(((it / NB) & 1) ^ 1), abort_flag,
                                  a.d_err, 6, wait_ns);
                    if (!ok) break;
                    tc::fence_after_sync();
                    const uint32_t d1 = tmem + (uint32_t)(b * BN);
                    const uint32_t st = ring_lo + (uint32_t)(s * (C::stage_bytes >> 4));
                    constexpr uint32_t H = tc::DESC_HI;
                    if (PERSAMPLE) {
#pragma unroll
                        for (int sl = 0; sl < KS; ++sl) {
                            const uint64_t da = tc::desc_of(ax + sl * 256, H);
                            const uint64_t db = tc::desc_of(st + ((C::tex_off + sl * 4096) >> 4), H);
                            if (TEX8)
                                tc::mma_fp8(d1, da, db, C::id_tex, sl > 0);
                            else
                                tc::mma_bf16(d1, da, db, C::id_tex, sl > 0);
                        }
                    }
                    tc::mma_bf16(d1, tc::desc_of(ap, H), tc::desc_of(st + (C::col_off >> 4), H),
                                 C::id_bf16, (PERSAMPLE && KS > 0) ? 1 : 0);
                    tc::mma_bf16(d1, tc::desc_of(ap + 256, H), tc::desc_of(st + (C::l0_off >> 4), H),
                                 C::id_bf16, 1);
                    tc::mma_bf16(d1, tc::desc_of(ap + 512, H),
                                 tc::desc_of(st + (C::l1_off >> 4) + tc::DESC_HALVES_LBO,
                                             tc::DESC_HALVES_HI),
                                 C::id_bf16, 1);
                    if (!ONE_COMMIT) tc::mma_commit(empty + s);
                    tc::mma_commit(tmem_full + b);
                    last = it;
                }
                if (!ok) break;
                tc::mma_commit(acol_empty + cb);
                ok = next_num(rp, num, true);
                if (!ok) break;
                const Item nxt = item_of(a, num);
                if (nxt.img < 0 || nxt.img != itm.img || nxt.pt != itm.pt)
                    tc::mma_commit(atex_empty + (int)((ptc - 1) % ATB));
                itm = nxt;
                ++li;
            }
            // drain: the last MMAs must finish before the tensor memory is freed
            if (last >= 0)
                tc::mbar_wait(tmem_full + (int)(last % NB), (uint32_t)((last / NB) & 1),
                              tc::globaltimer() + wait_ns);
        }
    } else {
        // ------------------------------------------------------------ epilogue
        const int q = warp & 3, hf = warp >> 2;  // lane quadrant, column part
        const int r = 32 * q + lane;             // pixel row of the tile
        const int rx = r % TW, ry = r / TW;
        // x' = position relative to the pixel tile's centre
        const int xpx = rx - TW / 2, xpy = ry - TH / 2;
        const float xsq = (float)(xpx * xpx + xpy * xpy);
        const float Cc = LOG2E / (2.f * a.sigma_c2);
        const float log_col_norm = 1.5f * logf(6.283185307179586f * a.sigma_c2);
        uint32_t it = 0, li = 0, pwr = 0;  // tiles, items, pixel-tile operands written
        bool ok = true;

        // co-support words a pixel row holds in registers (Wk <= WKM)
        constexpr int WKM = !PERSAMPLE ? 1 : TEX8 ? KS + 1 : KS / 2 + 1;
        struct Px {
            bool live;
            int pix;
            float IR, IG, IB, I2;
            int popx;
            int D;             // squared scribble distance of the item's label
            uint32_t bw[WKM];  // this pixel's co-support words
        };
        // an item's pixel row: the loads are issued here and used only after
        // the current item's first tile (px_finish), so that their latency
        // hides behind it
        auto px_issue = [&](const TcImage& im, int pt, int lab) {
            Px p;
            const int x = (pt % im.ntx) * TW + rx, y = (pt / im.ntx) * TH + ry;
            p.live = x < im.W && y < im.H;
            p.pix = p.live ? y * im.W + x : 0;  // < 2^31 (side <= 23170)
            const float* Ip = im.img + (size_t)p.pix * 3;
            p.IR = Ip[0];
            p.IG = Ip[1];
            p.IB = Ip[2];
            const uint32_t* bxp = im.bitmask + (size_t)p.pix * a.Wk;
#pragma unroll
            for (int w = 0; w < WKM; ++w) p.bw[w] = PERSAMPLE && w < a.Wk ? bxp[w] : 0u;
            p.D = p.live ? im.dist2[(size_t)lab * ((long long)im.H * im.W) + p.pix] : 0;
            return p;
        };
        auto px_finish = [&](Px& p) {
            p.I2 = fmaf(p.IR, p.IR, fmaf(p.IG, p.IG, p.IB * p.IB));
            p.popx = 0;
#pragma unroll
            for (int w = 0; w < WKM; ++w) p.popx += p.live ? __popc(p.bw[w]) : 0;
        };
        // texture operand rows of a pixel tile (the codes of the MMA slabs):
        // this warp writes slabs sl = hf, hf + EPQ, ... of buffer pwr % ATB
        auto write_atex = [&](const Px& p) {
            // the factorised form has no texture operand: only the arrival,
            // which orders the pixel tiles for the MMA issuer
            if (PERSAMPLE) {
            const bool wok = spin_warp(atex_empty + (int)(pwr % ATB),
                                       (uint32_t)(((pwr / ATB) & 1) ^ 1), abort_flag, a.d_err, 7,
                                       wait_ns);
            if (!wok) return false;
            uint8_t* ax = atex + (int)(pwr % ATB) * C::tex_bytes;
            for (int sl = hf; sl < KS; sl += EPQ) {
                // FP8: slab sl holds codes 32 sl .. 32 sl + 31 (bitmask word sl);
                // BF16: codes 16 sl .. 16 sl + 15 (half of word sl / 2)
                const int wi = TEX8 ? sl : sl >> 1;
                uint32_t word = 0u;
#pragma unroll
                for (int w = 0; w < WKM; ++w) word = w == wi ? p.bw[w] : word;
                if (!p.live) word = 0u;
                const int j0 = TEX8 ? 32 * sl : 16 * sl;
                const int valid = p.live ? min(max(a.k - j0, 0), TEX8 ? 32 : 16) : 0;
                const uint32_t bits = TEX8 ? word : (word >> (16 * (sl & 1))) & 0xFFFFu;
                uint32_t wv[8];
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    uint32_t packed = 0;
                    if (TEX8) {
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const int jj = 4 * c + e;
                            const uint32_t v = jj < valid ? (((bits >> jj) & 1u) ? 0x38u : 0xB8u) : 0u;
                            packed |= v << (8 * e);
                        }
                    } else {
#pragma unroll
                        for (int e = 0; e < 2; ++e) {
                            const int jj = 2 * c + e;
                            const uint32_t v = jj < valid ? (((bits >> jj) & 1u) ? 0x3F80u : 0xBF80u) : 0u;
                            packed |= v << (16 * e);
                        }
                    }
                    wv[c] = packed;
                }
                uint8_t* base = ax + sl * 4096;
                *reinterpret_cast<uint4*>(base + tc::slab_off(r, 0)) = make_uint4(wv[0], wv[1], wv[2], wv[3]);
                *reinterpret_cast<uint4*>(base + tc::slab_off(r, 16)) = make_uint4(wv[4], wv[5], wv[6], wv[7]);
            }
            tc::fence_proxy_async_smem();
            }
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(atex_full + (int)(pwr % ATB));
            ++pwr;
            return true;
        };
        // pixel-side operand rows of item number n (label lab at the pixel
        // tile of p): colour (16 bf16, two halves) and location L0, L1
        // (pieces of -f x' and f, f = nA / Bt, matching the sample side's
        // pieces of 2u and |u|^2, then +-1 for the texture codes that ride in
        // L1); jobs 0..3 = colour half 0, colour half 1, L0, L1, job j on
        // warp part j % EPQ
        auto write_acol = [&](const Px& p, uint32_t n) {
            const int cb = (int)(n & 1);
            const bool wok = spin_warp(acol_empty + cb, (uint32_t)(((n >> 1) & 1) ^ 1), abort_flag,
                                       a.d_err, 8, wait_ns);
            if (!wok) return false;
            const int D = p.D;
            const float rho = a.alpha * fmaxf(sqrtf((float)D), a.d_min);
            const float s2 = a.rho_var ? rho : rho * rho;  // location variance
            const float nA = -LOG2E / (2.f * s2);
            const float g = PERSAMPLE ? (a.kappa_beta * rho) / LOG2E : 1.f;
            const float f = nA * g;
            uint8_t* ap = acol + cb * C::AP;
#pragma unroll
            for (int job = hf; job < 4; job += EPQ) {
                uint4 lo = make_uint4(0, 0, 0, 0), hi = make_uint4(0, 0, 0, 0);
                if (job < 2) {
                    uint16_t h0, l0, h1, l1;
                    if (job == 0) {
                        split_bf16(2.f * Cc * g * p.IR, h0, l0);
                        split_bf16(2.f * Cc * g * p.IG, h1, l1);
                    } else {
                        split_bf16(2.f * Cc * g * p.IB, h0, l0);
                        split_bf16(g, h1, l1);
                    }
                    lo = make_uint4(pack2(h0, h0), pack2(l0, l0), pack2(h1, h1), pack2(l1, l1));
                } else {
                    uint16_t f1, f2, f3;
                    split3_bf16(f, f1, f2, f3);
                    if (job == 2) {
                        uint16_t x1, x2, x3, y1, y2, y3;
                        split3_bf16(-f * (float)xpx, x1, x2, x3);
                        split3_bf16(-f * (float)xpy, y1, y2, y3);
                        lo = make_uint4(pack2(x1, x1), pack2(x2, x2), pack2(x3, x3), pack2(y1, y1));
                        hi = make_uint4(pack2(y2, y2), pack2(y3, y3), pack2(f1, f1), pack2(f1, f1));
                    } else {
                        // texture codes 32 KS + e (16 KS + e): +-1 for e < ext
                        uint32_t sg[EXT_MAX];
#pragma unroll
                        for (int e = 0; e < EXT_MAX; ++e) {
                            const int code = (TEX8 ? 32 : 16) * KS + e;
                            uint32_t word = 0u;
#pragma unroll
                            for (int w = 0; w < WKM; ++w) word = w == (code >> 5) ? p.bw[w] : word;
                            sg[e] = (PERSAMPLE && e < a.ext)
                                        ? (((word >> (code & 31)) & 1u) ? 0x3F80u : 0xBF80u)
                                        : 0u;
                        }
                        // L1 = [f2 f2 f2 f3 f3 0 0 0 | codes], against the sample
                        // side's [q0 q1 q2 q0 q1 0 0 0 | b0 .. b7]
                        lo = make_uint4(pack2(f2, f2), pack2(f2, f3), f3, 0u);
                        hi = make_uint4(sg[0] | (sg[1] << 16), sg[2] | (sg[3] << 16),
                                        sg[4] | (sg[5] << 16), sg[6] | (sg[7] << 16));
                    }
                }
                if (!p.live) lo = hi = make_uint4(0, 0, 0, 0);
                if (job < 2) {
                    *reinterpret_cast<uint4*>(ap + tc::slab_off(r, 16 * job)) = lo;
                } else {
                    uint8_t* sl = ap + 4096 * (job - 1);
                    *reinterpret_cast<uint4*>(sl + tc::slab_off(r, 0)) = lo;
                    *reinterpret_cast<uint4*>(sl + tc::slab_off(r, 16)) = hi;
                }
            }
            tc::fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(acol_full + cb);
            return true;
        };

        RingPos rp;
        int num = -1;
        ok = next_num(rp, num, false);
        Item itm = item_of(a, num);
        Px cpx{};
        if (ok && itm.img >= 0) {
            cpx = px_issue(a.images[itm.img], itm.pt, itm.lab);
            px_finish(cpx);
            ok = write_atex(cpx) && write_acol(cpx, 0);
        }
        while (ok && itm.img >= 0) {
            const TcImage& im = a.images[itm.img];
            const long long P = (long long)im.H * im.W;
            const int i = itm.lab;
            const float rho = a.alpha * fmaxf(sqrtf((float)cpx.D), a.d_min);
            const float s2 = a.rho_var ? rho : rho * rho;  // location variance
            const float nA = -LOG2E / (2.f * s2);
            const float Bt = PERSAMPLE ? LOG2E / (a.kappa_beta * rho) : 1.f;
            const float R0 = (PERSAMPLE ? -Bt * (float)cpx.popx : 0.f) - Cc * cpx.I2;
            const uint64_t bt2 = pk2(Bt, Bt);
            const int m_i = im.label_off[i + 1] - im.label_off[i];
            const float shift = (float)(96 - (32 - __clz(m_i - 1)));  // 96 - ceil(log2 m)
            // e_j = Bt D1_j + nA |x'|^2 + R0 (+ shift)
            const float R0x = fmaf(nA, xsq, R0);
            const uint64_t k2 = pk2(R0x + shift, R0x + shift);
            const int nt = tiles_of(im.tile_off, i);
            // the next item, and its pixel row's loads in flight during tile 0
            ok = next_num(rp, num, false);
            if (!ok) break;
            const Item nxt = item_of(a, num);
            const bool n_newpt = nxt.img >= 0 && (nxt.img != itm.img || nxt.pt != itm.pt);
            Px npx = cpx;
            if (n_newpt) {
                npx = px_issue(a.images[nxt.img], nxt.pt, nxt.lab);
            } else if (nxt.img >= 0) {
                npx.D = cpx.live ? im.dist2[(size_t)nxt.lab * P + cpx.pix] : 0;
            }
            float S = 0.f, Ccomp = 0.f;
            for (int t = 0; t < nt; ++t, ++it) {
                const int b = (int)(it % NB);
                ok = spin_warp(tmem_full + b, (uint32_t)((it / NB) & 1), abort_flag, a.d_err, 10,
                               wait_ns);
                if (!ok) break;
                tc::fence_after_sync();
                const int nvalid = min(BN, m_i - t * BN);
                const int cbase = hf * CPW;
                const uint32_t lb = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * BN + cbase);
                uint64_t x1[8];
                bool released = false;
                if (cbase + CPW <= nvalid) {  // warp-uniform: all columns valid
                    float ts = 0.f;
#pragma unroll
                    for (int ch = 0; ch < CPW / 16; ++ch) {
                        tc::tmem_ld16_wait_pk(lb + 16u * ch, x1);
                        if (ch == CPW / 16 - 1) {
                            // the last chunk is in registers: release the
                            // accumulator before its arithmetic
                            tc::fence_before_sync();
                            tc::mbar_arrive_elect(tmem_empty + b);
                            released = true;
                        }
                        ts += sum16_full(x1, bt2, k2);
                    }
                    two_sum(ts, S, Ccomp);
                } else if (cbase < nvalid) {  // warp-uniform: the label's last tile
#pragma unroll
                    for (int ch = 0; ch < CPW / 16; ++ch) {
                        const int nv = nvalid - cbase - 16 * ch;
                        if (nv > 0) {  // warp-uniform
                            tc::tmem_ld16_wait_pk(lb + 16u * ch, x1);
                            const float ts = nv >= 16 ? sum16_full(x1, bt2, k2)
                                                      : sum16_part(x1, nv, bt2, k2);
                            two_sum(ts, S, Ccomp);
                        }
                    }
                }
                // tcgen05.wait::ld is warp-collective: every lane's loads are
                // complete here; one elected lane releases the buffer
                if (!released) {
                    tc::fence_before_sync();
                    tc::mbar_arrive_elect(tmem_empty + b);
                }
                if (t == 0 && nxt.img >= 0) {
                    // the next item's operands, while this item's MMAs run on
                    if (n_newpt) px_finish(npx);
                    if (n_newpt && ATB == 2) ok = write_atex(npx);
                    ok = ok && write_acol(npx, li + 1);
                    if (!ok) break;
                }
            }
            if (!ok) break;
            // merge the EPQ column parts of each pixel. XB = 2 NB exchange
            // buffers: a part can run at most NB sample tiles ahead of another
            // (tensor memory holds NB accumulators and every item has at least
            // one tile), so buffer li % XB is free when rewritten.
            const int xbuf = (int)(li % C::XB);
            float2* xb = xchg + (size_t)xbuf * (EPQ - 1) * 4 * 32;
            uint64_t* xbar = xchg_full + xbuf * 4 + q;
            if (hf > 0) {
                xb[((hf - 1) * 4 + q) * 32 + lane] = make_float2(S, Ccomp);
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(xbar);
            } else {
                ok = spin_warp(xbar, (uint32_t)((li / C::XB) & 1), abort_flag, a.d_err, 11, wait_ns);
                if (!ok) break;
                float Sm = S, Cm = Ccomp;
#pragma unroll
                for (int h = 0; h < EPQ - 1; ++h) {
                    const float2 v = xb[(h * 4 + q) * 32 + lane];
                    Sm += v.x;
                    Cm += v.y;
                }
                const float tot = Sm + Cm;  // shifted by 2^shift
                const float lse2 = log2f(tot) - shift;
                const float Lv = lse2 * LN2 - logf((float)m_i) - logf(6.283185307179586f * s2) -
                                 log_col_norm;
                // below the floor the FP32 terms may have lost mass to
                // underflow; above the tolerance the bound on the error of L
                // (log2 units) is too loose: recompute in FP64. Bound: colour
                // splits 2^-15 C Q. Accumulation of the colour and the two
                // location MMAs onto the exact texture sum, 2^-21 of the
                // magnitudes per instruction, plus the location pieces'
                // residuals (<= 2^-24): at most 2^-19 (Bt k + C Q + |nA| M_j),
                // where the location products of sample j sum in magnitude to
                // M_j <= (|u_j| + |x'|)^2 <= 2 |x - x_j|^2 + 8 |x'|^2 and
                // |nA| |x - x_j|^2 <= |e_j| (every part of the exponent is
                // <= 0); weighted by the pairs' shares of the sum, |e_j|
                // averages at most |log2 S| + log2 m. The FP32 epilogue: 6u
                // per pair on the same weights plus the per-pixel constant.
                const float im2 = im.imax2[i];
                const float CQ = Cc * fmaf(2.f * sqrtf(cpx.I2), sqrtf(im2), im2);
                const float BK = PERSAMPLE ? Bt * (float)a.k : 0.f;
                const float Ew = fabsf(lse2) + log2f((float)m_i);
                const float E2 = 3.1e-05f * CQ +
                                 1.9073486e-06f * (BK + CQ - 8.f * nA * xsq + 2.f * Ew) +
                                 3.5762787e-07f * (3.f * Ew + 2.f * fabsf(R0x) + shift + 1.f);
                const bool flag = !(tot >= FLOOR_PER_SAMPLE * (float)m_i) ||
                                  (a.l_tol > 0.f && E2 * LN2 > a.l_tol * fmaxf(fabsf(Lv), 1.f));
                if (cpx.live) {
                    // -L into the output plane; the label normalisation follows
                    // in its own pass once every row is written
                    im.neglog[(size_t)i * P + cpx.pix] = -Lv;
                    if (flag) {
                        // the FP64 recompute lists a pixel once, with all its flagged rows
                        const unsigned long long old =
                            atomicOr(a.flags + im.pix_off + cpx.pix, 1ull << i);
                        if (old == 0ull) {
                            const int idx = atomicAdd(a.fb_count, 1);
                            if (idx < a.fb_cap) a.fb_list[idx] = make_int4(itm.img, cpx.pix, 0, 0);
                        }
                    }
                }
            }
            // a new pixel tile's texture operand once this one is consumed
            if (n_newpt && ATB == 1) ok = write_atex(npx);
            itm = nxt;
            cpx = npx;
            ++li;
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, C::TMEM_COLS);
    }
}

// Recompute of the pixels flagged by the sum (a label row below the FP32
// floor or above the error tolerance): one warp per listed pixel, its
// flagged rows read from the per-pixel flag words. Each
// flagged label row is summed again with the exponents
// e_j = -|x - x_j|^2 / (2 rho^2) - |I - I_j|^2 / (2 sigma_c2) [- TSM / beta]
// formed in double precision (no cancellation between expanded products),
// their offsets from the row maximum exponentiated in FP32 (relative error
// ~1e-7 per term) and accumulated in double across the lanes (two passes:
// maximum, then sum); the other rows keep the sum's value. The label
// normalisation (and, factorised, the texture posterior) is then redone in
// double for the pixel.
__global__ void __launch_bounds__(128) refine_fp64_kernel(
    const TcImage* __restrict__ images, const int4* __restrict__ list,
    const int* __restrict__ count, int cap, const unsigned long long* __restrict__ flags, int Wk,
    double alpha, double d_min, double kappa_beta, double sigma_c2, bool persample, bool rho_var,
    int* __restrict__ d_err) {
    __shared__ double sL[4][CS_MAX_LABELS];
    __shared__ double sT[4][CS_MAX_LABELS];
    int cnt = *count;
    if (cnt > cap) {
        if (blockIdx.x == 0 && threadIdx.x == 0 && atomicCAS(d_err, 0, CS_DEVERR_REFINE_FULL) == 0)
            d_err[1] = cnt;
        cnt = cap;
    }
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int nwarps = gridDim.x * 4;
    const double PI2 = 6.283185307179586;
    const double col_norm = 1.5 * log(PI2 * sigma_c2), c_col = 0.5 / sigma_c2;
    for (int e = blockIdx.x * 4 + wib; e < cnt; e += nwarps) {
        const int4 it = list[e];
        const TcImage& im = images[it.x];
        const int pix = it.y, x = pix % im.W, y = pix / im.W;
        const uint64_t fmask = flags[im.pix_off + pix];  // the pixel's flagged label rows
        const long long P = (long long)im.H * im.W;
        const double IR = im.img[(size_t)pix * 3], IG = im.img[(size_t)pix * 3 + 1],
                     IB = im.img[(size_t)pix * 3 + 2];
        uint32_t bx[8];
#pragma unroll
        for (int w = 0; w < 8; ++w) bx[w] = w < Wk ? im.bitmask[(size_t)pix * Wk + w] : 0u;
        for (int i = 0; i < im.n_labels; ++i) {
            const double rho = alpha * fmax(sqrt((double)im.dist2[(size_t)i * P + pix]), d_min);
            if (lane == 0 && !persample && im.rep) {
                int h = 0;
                for (int w = 0; w < Wk; ++w) h += __popc(bx[w] ^ im.rep[i * Wk + w]);
                sT[wib][i] = -(double)h / (kappa_beta * rho);
            }
            if (!((fmask >> i) & 1ull)) {  // this row keeps the sum's value
                if (lane == 0) sL[wib][i] = -(double)im.neglog[(size_t)i * P + pix];
                continue;
            }
            const double s2 = rho_var ? rho : rho * rho;  // location variance
            const double c_loc = 0.5 / s2;
            const double c_tex = persample ? 1.0 / (kappa_beta * rho) : 0.0;
            const int off = im.label_off[i], m = im.label_off[i + 1] - off;
            auto expo = [&](int j) {
                const int s = off + j;
                const double dx = (double)x - (double)im.sx[s], dy = (double)y - (double)im.sy[s];
                const double dr = IR - (double)im.sr[s], dg = IG - (double)im.sg[s],
                             db = IB - (double)im.sb[s];
                int h = 0;
                if (persample)
                    for (int w = 0; w < Wk; ++w) h += __popc(bx[w] ^ im.sbits[(size_t)w * im.n_samples + s]);
                return -(dx * dx + dy * dy) * c_loc - (dr * dr + dg * dg + db * db) * c_col -
                       (double)h * c_tex;
            };
            double mx = -INFINITY;
            for (int j = lane; j < m; j += 32) mx = fmax(mx, expo(j));
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            double sum = 0.0;
            for (int j = lane; j < m; j += 32) sum += (double)__expf((float)(expo(j) - mx));
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
            if (lane == 0)
                sL[wib][i] = mx + log(sum) - log((double)m) - log(PI2 * s2) - col_norm;
        }
        __syncwarp();
        if (lane == 0) {
            const int n = im.n_labels;
            if (!persample && im.rep) {
                double tm = -INFINITY, ts = 0.0;
                for (int i = 0; i < n; ++i) tm = fmax(tm, sT[wib][i]);
                for (int i = 0; i < n; ++i) ts += exp(sT[wib][i] - tm);
                const double tl = tm + log(ts);
                for (int i = 0; i < n; ++i) sL[wib][i] += sT[wib][i] - tl;
            }
            double lm = -INFINITY, ls = 0.0;
            for (int i = 0; i < n; ++i) lm = fmax(lm, sL[wib][i]);
            for (int i = 0; i < n; ++i) ls += exp(sL[wib][i] - lm);
            const double lse = lm + log(ls);
            for (int i = 0; i < n; ++i) {
                im.neglog[(size_t)i * P + pix] = (float)(-sL[wib][i]);
                if (im.post) im.post[(size_t)i * P + pix] = (float)exp(sL[wib][i] - lse);
            }
        }
        __syncwarp();
    }
}

// Morton order of each label's samples in chunks of 4096 (one block per
// chunk, bitonic sort of (key, index) pairs in shared memory): consecutive
// 128-sample tiles then cover compact regions.
__device__ __forceinline__ uint32_t morton16(uint32_t v) {
    v &= 0xFFFFu;
    v = (v | (v << 8)) & 0x00FF00FFu;
    v = (v | (v << 4)) & 0x0F0F0F0Fu;
    v = (v | (v << 2)) & 0x33333333u;
    v = (v | (v << 1)) & 0x55555555u;
    return v;
}

__global__ void __launch_bounds__(1024) morton_sort_kernel(const int32_t* __restrict__ label_off,
                                                           int n_labels,
                                                           const int32_t* __restrict__ sample_pix,
                                                           int W, long long P,
                                                           int32_t* __restrict__ perm) {
    __shared__ uint32_t key[4096];
    __shared__ int32_t idx[4096];
    // chunk -> (label, first sample, count)
    int b = blockIdx.x, i = 0, start = 0, cnt = 0;
    for (; i < n_labels; ++i) {
        const int m = label_off[i + 1] - label_off[i];
        const int nch = (m + 4095) / 4096;
        if (b < nch) {
            start = label_off[i] + b * 4096;
            cnt = min(4096, label_off[i + 1] - start);
            break;
        }
        b -= nch;
    }
    if (i == n_labels) return;
    int n2 = 1;
    while (n2 < cnt) n2 <<= 1;
    for (int e = threadIdx.x; e < n2; e += blockDim.x) {
        if (e < cnt) {
            const int sidx = start + e;
            int pix = sample_pix[sidx];
            if (pix < 0 || pix >= P) pix = 0;  // reported by the seed kernel
            key[e] = morton16((uint32_t)(pix % W)) | (morton16((uint32_t)(pix / W)) << 1);
            idx[e] = sidx;
        } else {
            key[e] = 0xFFFFFFFFu;
            idx[e] = 0x7FFFFFFF;
        }
    }
    __syncthreads();
    for (int kk = 2; kk <= n2; kk <<= 1)
        for (int jj = kk >> 1; jj > 0; jj >>= 1) {
            for (int e = threadIdx.x; e < n2; e += blockDim.x) {
                const int partner = e ^ jj;
                if (partner > e) {
                    const bool up = (e & kk) == 0;
                    const uint32_t ka = key[e], kb = key[partner];
                    const int ia = idx[e], ib = idx[partner];
                    const bool gt = ka > kb || (ka == kb && ia > ib);
                    if (gt == up) {
                        key[e] = kb;
                        key[partner] = ka;
                        idx[e] = ib;
                        idx[partner] = ia;
                    }
                }
            }
            __syncthreads();
        }
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) perm[start + e] = idx[e];
}

// Sample tiles laid out as the bulk-copied part of a ring stage: the
// second half of the location slab L1 (the sample's texture codes beyond
// the texture slabs, code 32 KS + e or 16 KS + e as bf16 1 / 0 in column
// 8 + e), the texture slabs (b_j in {0, 1}) and the colour slab (hi/lo bf16
// of I_j and of -C |I_j|^2); padded rows are zero. tile_xy receives each
// tile slot's sample position x | y << 16, from which the producer forms
// the location rows per pixel tile.
template <bool TEX8, int KS, bool PERSAMPLE>
__global__ void build_tiles_kernel(const int32_t* __restrict__ label_off,
                                   const int32_t* __restrict__ tile_off, int n_labels,
                                   int total_tiles, SampleTables t, int n_samples, int k,
                                   float Cc, const int32_t* __restrict__ perm,
                                   uint8_t* __restrict__ blob, uint32_t* __restrict__ tile_xy,
                                   float* __restrict__ imax2,
                                   TcImage desc, TcImage* __restrict__ desc_dst) {
    using C = Cfg<TEX8, KS, PERSAMPLE>;
    const long long gid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (gid == 0) *desc_dst = desc;  // this image's descriptor for the sum launch
    if (gid >= (long long)total_tiles * BN) return;
    const int tile = (int)(gid / BN), r = (int)(gid % BN);
    int lo = 0, hi = n_labels - 1;  // label of this tile
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tile_off[mid] <= tile) lo = mid; else hi = mid - 1;
    }
    const int i = lo;
    const int first = label_off[i] + (tile - tile_off[i]) * BN;
    const int pos = first + r;
    const bool valid = pos < label_off[i + 1];
    const int s = valid ? perm[pos] : 0;
    tile_xy[gid] = valid ? (uint32_t)t.sx[s] | ((uint32_t)t.sy[s] << 16) : 0u;
    // the bulk-copied part starts with L1's second half
    uint8_t* cp = blob + (size_t)tile * C::copy_bytes;
    uint32_t xw[4] = {0u, 0u, 0u, 0u};
    if (PERSAMPLE && valid)
        for (int e = 0, j = (TEX8 ? 32 : 16) * KS; j < k && e < EXT_MAX; ++e, ++j)
            if ((t.sbits[(size_t)(j >> 5) * n_samples + s] >> (j & 31)) & 1u)
                xw[e >> 1] |= 0x3F80u << (16 * (e & 1));
    *reinterpret_cast<uint4*>(cp + tc::halves_off(r, 0)) = make_uint4(xw[0], xw[1], xw[2], xw[3]);
    uint8_t* st = cp + (C::tex_off - C::copy_off);
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
    uint32_t pw[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (valid) {
        const float R = t.sr[s], G = t.sg[s], B = t.sb[s];
        const float i2 = fmaf(R, R, fmaf(G, G, B * B));
        atomicMax(reinterpret_cast<int*>(imax2) + i, __float_as_int(i2));  // i2 >= 0
        const float qv = -Cc * i2;
        uint16_t hr, lr, hg, lg, hb, lb, hq, lq;
        split_bf16(R, hr, lr);
        split_bf16(G, hg, lg);
        split_bf16(B, hb, lb);
        split_bf16(qv, hq, lq);
        pw[0] = pack2(hr, lr); pw[1] = pack2(hr, lr);
        pw[2] = pack2(hg, lg); pw[3] = pack2(hg, lg);
        pw[4] = pack2(hb, lb); pw[5] = pack2(hb, lb);
        pw[6] = pack2(hq, lq); pw[7] = pack2(hq, lq);
    }
    uint8_t* sc = cp + (C::col_off - C::copy_off);
    *reinterpret_cast<uint4*>(sc + tc::slab_off(r, 0)) = make_uint4(pw[0], pw[1], pw[2], pw[3]);
    *reinterpret_cast<uint4*>(sc + tc::slab_off(r, 16)) = make_uint4(pw[4], pw[5], pw[6], pw[7]);
}

template <bool TEX8, int KS, bool PERSAMPLE>
cudaError_t tiles(const TcLaunch& L, cudaStream_t st) {
    const int total_tiles = L.total_tiles;
    const float Cc = 1.4426950408889634f / (2.f * L.sigma_c2);
    TcImage d{};
    d.img = L.img;
    d.bitmask = L.bitmask;
    d.dist2 = L.dist2;
    d.label_off = L.d_label_off;
    d.tile_off = L.d_tile_off;
    d.blob = L.blob;
    d.tile_xy = L.t.tile_xy;
    d.rep = L.t.rep;
    d.neglog = L.neglog;
    d.post = L.post;
    d.sx = L.t.sx;
    d.sy = L.t.sy;
    d.sr = L.t.sr;
    d.sg = L.t.sg;
    d.sb = L.t.sb;
    d.sbits = L.t.sbits;
    d.imax2 = L.imax2;
    d.n_samples = L.n_samples;
    d.H = L.H;
    d.W = L.W;
    d.ntx = (L.W + TW - 1) / TW;
    d.n_labels = L.n_labels;
    d.n_ptiles = tc_pixel_tiles(L.H, L.W);
    d.first_item = L.first_item;
    d.pix_off = L.pix_off;
    d.first_ptile = L.first_ptile;
    cudaError_t e = cudaMemsetAsync(L.imax2, 0, sizeof(float) * L.n_labels, st);
    if (e != cudaSuccess) return e;
    build_tiles_kernel<TEX8, KS, PERSAMPLE>
        <<<(unsigned)(((long long)total_tiles * BN + 127) / 128), 128, 0, st>>>(
            L.d_label_off, L.d_tile_off, L.n_labels, total_tiles, L.t, L.n_samples, L.k, Cc,
            L.t.perm, L.blob, L.t.tile_xy, L.imax2, d, L.desc);
    return cudaGetLastError();
}

template <bool TEX8, int KS, bool PERSAMPLE, bool SOLO>
cudaError_t sum(const TcImage* descs, int n_images, const TcSumParams& p, cudaStream_t st) {
    using C = Cfg<TEX8, KS, PERSAMPLE, SOLO>;
    static_assert(C::smem_bytes <= 227 * 1024, "shared memory budget");
    TcArgs a{};
    a.images = descs;
    a.n_images = n_images;
    a.n_items = p.n_items;
    a.total_pixels = p.total_pixels;
    a.k = p.k;
    a.Wk = (p.k + 31) / 32;
    a.ext = PERSAMPLE ? tex_ext(p.k, TEX8) : 0;
    a.alpha = p.alpha;
    a.d_min = p.d_min;
    a.kappa_beta = p.kappa_beta;
    a.sigma_c2 = p.sigma_c2;
    a.rho_var = p.rho_var;
    a.d_err = p.d_err;
    a.fb_list = p.fb_list;
    a.fb_count = p.fb_count;
    a.fb_cap = p.fb_cap;
    a.queue = p.queue;
    a.flags = p.flags;
    a.l_tol = p.l_tol;
    a.wait_ns = p.wait_ns;
    a.stall = p.stall;
    cudaError_t e = cudaFuncSetAttribute(sum_tc_kernel<TEX8, KS, PERSAMPLE, SOLO>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, C::smem_bytes);
    if (e == cudaSuccess) e = cudaMemsetAsync(p.fb_count, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(p.queue, 0, 2 * sizeof(unsigned), st);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(p.flags, 0, sizeof(unsigned long long) * (size_t)p.total_pixels, st);
    if (e != cudaSuccess) return e;
    const long long slots = (long long)C::MIN_BLOCKS * p.n_sm;
    const int grid = (int)(p.n_items < slots ? p.n_items : slots);
    // whole pixel tiles while more than about one per CTA is left, then
    // single items
    long long total_pt = 0;
    for (int g = 0; g < n_images; ++g) total_pt += p.shapes[g].x;
    const long long pt1 = total_pt > grid ? total_pt - grid : 0;
    long long i1 = 0, seen = 0;
    for (int g = 0; g < n_images && seen < pt1; ++g) {
        const long long take = p.shapes[g].x < pt1 - seen ? p.shapes[g].x : pt1 - seen;
        i1 += take * p.shapes[g].y;
        seen += take;
    }
    a.pt1 = (int)pt1;
    a.i1 = i1;
    sum_tc_kernel<TEX8, KS, PERSAMPLE, SOLO><<<grid, C::THREADS, C::smem_bytes, st>>>(a);
    refine_fp64_kernel<<<2 * p.n_sm, 128, 0, st>>>(
        descs, p.fb_list, p.fb_count, p.fb_cap, p.flags, (p.k + 31) / 32, (double)p.alpha,
        (double)p.d_min, (double)p.kappa_beta, (double)p.sigma_c2, PERSAMPLE, p.rho_var, p.d_err);
    const long long nblk = (p.total_pixels + 255) / 256, cap = 8ll * p.n_sm;
    normalise_kernel<PERSAMPLE><<<(unsigned)(nblk < cap ? nblk : cap), 256, 0, st>>>(a);
    return cudaGetLastError();
}

// Dispatch on (texture format, texture slabs, per-sample form).
template <class F>
cudaError_t dispatch(int k, bool tex8, bool persample, F&& f) {
    if (!tc_supported(k, tex8)) return cudaErrorInvalidValue;
    if (!persample) return f(std::integral_constant<bool, true>{}, std::integral_constant<int, 1>{},
                             std::integral_constant<bool, false>{});
    const int ks = tex_slabs(k, tex8);
#define CS_TC_CASE(N)                                                                        \
    case N:                                                                                  \
        return tex8 ? f(std::integral_constant<bool, true>{}, std::integral_constant<int, N>{}, \
                        std::integral_constant<bool, true>{})                                \
                    : f(std::integral_constant<bool, false>{}, std::integral_constant<int, N>{}, \
                        std::integral_constant<bool, true>{});
    switch (ks) {
        CS_TC_CASE(0)
        CS_TC_CASE(1)
        CS_TC_CASE(2)
        CS_TC_CASE(3)
        CS_TC_CASE(4)
        CS_TC_CASE(5)
        CS_TC_CASE(6)
        CS_TC_CASE(7)
        CS_TC_CASE(8)
        default: return cudaErrorInvalidValue;
    }
#undef CS_TC_CASE
}

}  // namespace

size_t tc_copy_bytes(int k, bool tex8, bool persample) {
    const int ks = tex_slabs(k, tex8);
    return 2048 + (size_t)(persample ? ks * 4096 : 0) + 4096;
}

int tc_tiles_per_label(int m) { return (m + BN - 1) / BN; }

int tc_tile_samples() { return BN; }

bool tc_supported(int k, bool tex8) { return tex8 ? k <= 256 : k <= 128; }

int tc_pixel_tiles(int H, int W) { return ((W + TW - 1) / TW) * ((H + TH - 1) / TH); }

cudaError_t launch_tc_sort(const TcLaunch& L, cudaStream_t st) {
    morton_sort_kernel<<<L.n_chunks, 1024, 0, st>>>(L.d_label_off, L.n_labels, L.sample_pix, L.W,
                                                    (long long)L.H * L.W, L.t.perm);
    return cudaGetLastError();
}

cudaError_t launch_tc_tiles(const TcLaunch& L, cudaStream_t st) {
    return dispatch(L.k, L.tex8, L.persample, [&](auto t8, auto ks, auto ps) {
        return tiles<decltype(t8)::value, decltype(ks)::value, decltype(ps)::value>(L, st);
    });
}

cudaError_t launch_tc_prepare(const TcLaunch& L, cudaStream_t st) {
    cudaError_t e = launch_tc_sort(L, st);
    return e != cudaSuccess ? e : launch_tc_tiles(L, st);
}

cudaError_t launch_tc_sum(const TcImage* descs, int n_images, const TcSumParams& p,
                          cudaStream_t st) {
    if (n_images < 1 || p.n_items < 1 || p.n_items >= (1ll << 31)) return cudaErrorInvalidValue;
    return dispatch(p.k, p.tex8, p.persample, [&](auto t8, auto ks, auto ps) {
        constexpr bool T8 = decltype(t8)::value, PS = decltype(ps)::value;
        constexpr int K = decltype(ks)::value;
        return p.variant == 1 ? sum<T8, K, PS, true>(descs, n_images, p, st)
                              : sum<T8, K, PS, false>(descs, n_images, p, st);
    });
}

bool tc_sum_shape(int k, bool tex8, bool persample, int variant, int* shape) {
    return dispatch(k, tex8, persample, [&](auto t8, auto ks, auto ps) {
               constexpr bool T8 = decltype(t8)::value, PS = decltype(ps)::value;
               constexpr int K = decltype(ks)::value;
               using C0 = Cfg<T8, K, PS, false>;
               using C1 = Cfg<T8, K, PS, true>;
               const bool solo = variant == 1;
               shape[0] = solo ? C1::MIN_BLOCKS : C0::MIN_BLOCKS;
               shape[1] = solo ? C1::STAGES : C0::STAGES;
               shape[2] = solo ? C1::ATB : C0::ATB;
               shape[3] = solo ? C1::EPI_WARPS : C0::EPI_WARPS;
               return cudaSuccess;
           }) == cudaSuccess;
}

cudaError_t launch_sum_tc_prepare(const TcLaunch& L, bool sorted, cudaStream_t st) {
    TcLaunch one = L;
    one.first_item = 0;
    one.pix_off = 0;
    one.first_ptile = 0;
    return sorted ? launch_tc_tiles(one, st) : launch_tc_prepare(one, st);
}

cudaError_t launch_sum_tc_run(const TcLaunch& L, cudaStream_t st) {
    TcSumParams p{L.k,       L.tex8,  L.persample, L.alpha,      L.d_min, L.kappa_beta,
                  L.sigma_c2, L.d_err, L.n_sm,      L.fb_list,    L.fb_count,
                  L.H * L.W,  L.l_tol, L.rho_var,   L.wait_ns,    L.stall};
    const int npt = tc_pixel_tiles(L.H, L.W);
    p.n_items = (long long)npt * L.n_labels;
    p.total_pixels = (long long)L.H * L.W;
    const int2 shape = make_int2(npt, L.n_labels);
    p.shapes = &shape;
    p.queue = L.queue;
    p.flags = L.flags;
    return launch_tc_sum(L.desc, 1, p, st);
}
