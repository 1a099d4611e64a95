// Learned surrogate of the data term on the tensor cores: an
// nin -> 64 -> 64 -> 64 -> n MLP (SiLU) that predicts, per pixel and label,
// the log kernel sum
//   T_i(x) = log sum_j k_rho(x - x_ij) k_sigma(I - I_ij) [exp(-TSM / beta)]
// of Sec. 3.1 (Eq. color, Eq. post_text); L_i then follows exactly from the
// scribble distance transform (and, in the factorised mode, the exact
// texture posterior of Eq. post_text).
//
// Parameter vector (fp32 masters), nin inputs, n labels:
//   W1 [64][nin] | b1 [64] | W2 [64][64] | b2 [64] | W3 [64][64] | b3 [64] | W4 [n][64] | b4 [n]
// The kernels use the weights rounded to bf16.
//
// Every contraction runs on tcgen05 (kind::f16, bf16 operands, fp32
// accumulation in tensor memory), 128 rows (pixels or training rows) per
// tile, one thread per row for the element-wise work:
//   forward   Z_l = H_{l-1} W_l^T with H = hi + lo, two bf16 pieces of the
//             fp32 activation (hi = bf16(h), lo = bf16(h - hi)), so the
//             activations keep about 16 bits;
//   backward  P_{l-1} = D_l W_l with D = dLoss/dZ_l split the same way, and
//             the weight gradient dW_l = D_l^T H_{l-1} from the hi pieces of
//             H (D in both pieces), summed over the rows of the tile.
// Operands live in shared memory in one "row layout": element (r, c) of a
// tile with R rows at byte (c / 8) * 16 R + 16 r + 2 (c % 8). Read K-major
// (K = columns) it feeds the forward and the propagation's A operand; read
// MN-major (K = rows) the same bytes feed the weight gradient's operands and
// the propagation's B operand (W itself, not a transposed copy).
//
// Kernels
//   mlp_train_kernel  forward and backward over the CTA's tiles of a
//                     minibatch; per-CTA gradient sums (and loss) to a
//                     partials buffer, in a fixed order.
//   reduce_adam_kernel sums the partials over the CTAs (fixed order), then
//                     optionally takes a bias-corrected Adam step.
//   mlp_fwd_kernel<ROWS>  forward pass on given standardised rows.
//   mlp_fwd_kernel<EVAL>  features from the pixel, forward pass, then
//                     L_i = sd_t,i z_i + mu_t,i - log m_i - log(2 pi s2_i)
//                           - 1.5 log(2 pi sigma_c2) (+ the factorised
//                     texture log-posterior), the posteriors, and the fallback
//                     decision of the fallback rule (top-2 posterior margin
//                     below `margin`; under the guaranteed rule also a top-2
//                     gap below the calibrated gap_min): such pixels are
//                     listed for the exact sum to overwrite.
#include <cuda_bf16.h>

#include <cstdint>

#include "internal.h"
#include "tc_ptx.cuh"

namespace {

constexpr int HID = 64;
constexpr int TR = 128;   // rows per tile (the MMA's M)
constexpr int NTH = 256;  // threads per CTA, two per row
constexpr uint64_t MLP_WAIT_NS = 1000000000ull;

struct Dims {
    int nin, K0, n, NOp;
};
__host__ __device__ inline Dims dims_of(int nin, int n) {
    return Dims{nin, nin <= 32 ? 32 : 64, n, (n + 15) & ~15};
}

struct Off {
    int W1, b1, W2, b2, W3, b3, W4, b4, np;
};
__host__ __device__ inline Off off_of(int nin, int n) {
    Off o;
    o.W1 = 0;
    o.b1 = HID * nin;
    o.W2 = o.b1 + HID;
    o.b2 = o.W2 + HID * HID;
    o.W3 = o.b2 + HID;
    o.b3 = o.W3 + HID * HID;
    o.W4 = o.b3 + HID;
    o.b4 = o.W4 + n * HID;
    o.np = o.b4 + n;
    return o;
}

// ------------------------------------------------------------------ operand helpers
// Shared-memory descriptor with explicit leading / stride byte offsets (no swizzle).
__device__ __forceinline__ uint64_t sdesc(const void* p, uint32_t lbo, uint32_t sbo) {
    const uint32_t a = tc::smem_u32(p);
    uint64_t d = (uint64_t)((a & 0x3FFFFu) >> 4);
    d |= (uint64_t)(lbo >> 4) << 16;
    d |= (uint64_t)(sbo >> 4) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}
// Row-layout tile of R rows read K-major (K = columns): the next 8 columns
// are 16 R bytes on, the next 8 rows 128 bytes on.
__device__ __forceinline__ uint64_t desc_k(const void* p, uint32_t R) { return sdesc(p, 16u * R, 128u); }
// The same tile read MN-major (MN = columns, K = rows): the next 8 rows (K)
// are 128 bytes on, the next 8 columns (MN) 16 R bytes on.
__device__ __forceinline__ uint64_t desc_mn(const void* p, uint32_t R) { return sdesc(p, 128u, 16u * R); }
constexpr uint32_t A_MN = 1u << 15;  // instruction descriptor: A read MN-major
constexpr uint32_t B_MN = 1u << 16;  // instruction descriptor: B read MN-major

__device__ __forceinline__ uint32_t pack_bf2(float a, float b) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&h);
}
__device__ __forceinline__ float bf_hi(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

// The weights as the kernels read them (the "image"): the bf16 row-layout
// tiles W1 (64 x K0), W2, W3 (64 x 64), W4 (NOp x 64), zero outside the
// parameters, then the biases b1 b2 b3 b4 (64 fp32 each, bf16-rounded, b4
// zero beyond n). Built by pack_kernel, rewritten by every Adam step, and
// copied into shared memory in two bulk copies.
__host__ __device__ inline uint32_t img_wbytes(int K0, int NOp) {
    return 2u * HID * K0 + 4u * HID * HID + 2u * NOp * HID;
}
__host__ __device__ inline uint32_t img_bytes(int K0, int NOp) { return img_wbytes(K0, NOp) + 4u * 4 * HID; }

// Image element (bf16 index) of weight (r, c) of layer l, for a tile of R rows.
__host__ __device__ inline uint32_t img_elem(uint32_t tile0, uint32_t R, int r, int c) {
    return tile0 + (uint32_t)(c >> 3) * 8u * R + 8u * r + (c & 7);
}

// Bulk copy of the image into shared memory (thread 0 issues; every thread
// waits, bounded).
__device__ bool load_image(const unsigned char* img, uint32_t wbytes, unsigned char* w_dst,
                           float* bias_dst, uint64_t* bar, uint64_t wait_ns, int* d_err, int site) {
    if (threadIdx.x == 0) {
        tc::mbar_arrive_expect_tx(bar, wbytes + 4u * 4 * HID);
        tc::bulk_g2s(w_dst, img, wbytes, bar);
        tc::bulk_g2s(bias_dst, img + wbytes, 4u * 4 * HID, bar);
    }
    bool ok = true;
    uint64_t deadline = 0;
    for (uint32_t n = 0;; ++n) {
        if (tc::mbar_try_wait(bar, 0, 1000u)) break;
        if ((n & 63u) == 63u) {
            const uint64_t now = tc::globaltimer();
            if (deadline == 0) deadline = now + wait_ns;
            else if (now > deadline) {
                ok = false;
                break;
            }
        }
    }
    ok = __syncthreads_and(ok);
    if (!ok && threadIdx.x == 0 && atomicCAS(d_err, 0, CS_DEVERR_TIMEOUT) == 0) d_err[1] = site;
    return ok;
}

// Parameter i (value v) into its place in the image.
__device__ void img_store(unsigned char* img, const Off& of, const Dims& dm, int i, float v) {
    __nv_bfloat16* w = reinterpret_cast<__nv_bfloat16*>(img);
    float* bias = reinterpret_cast<float*>(img + img_wbytes(dm.K0, dm.NOp));
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    const uint32_t t2 = HID * dm.K0, t3 = t2 + HID * HID, t4 = t3 + HID * HID;
    if (i < of.b1) w[img_elem(0, HID, i / dm.nin, i % dm.nin)] = h;
    else if (i < of.W2) bias[i - of.b1] = __bfloat162float(h);
    else if (i < of.b2) w[img_elem(t2, HID, (i - of.W2) / HID, (i - of.W2) % HID)] = h;
    else if (i < of.W3) bias[HID + i - of.b2] = __bfloat162float(h);
    else if (i < of.b3) w[img_elem(t3, HID, (i - of.W3) / HID, (i - of.W3) % HID)] = h;
    else if (i < of.W4) bias[2 * HID + i - of.b3] = __bfloat162float(h);
    else if (i < of.b4) w[img_elem(t4, dm.NOp, (i - of.W4) / HID, (i - of.W4) % HID)] = h;
    else bias[3 * HID + i - of.b4] = __bfloat162float(h);
}

// Thread layout of a CTA (256 threads): warp w reads the tensor-memory lanes
// 32 (w % 4) .. 32 (w % 4) + 31, i.e. those rows of the tile, and owns
// columns 32 (w / 4) .. 32 (w / 4) + 31 of its row: two threads per row.

// Columns [c0, c0 + 32) of row r, clipped to C (a multiple of 8), into a
// 128-row tile as the hi and (optionally) lo bf16 pieces, 16-byte stores.
__device__ __forceinline__ void put_half(const float (&v)[32], int c0, int C, unsigned char* hi,
                                         unsigned char* lo, int r) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int c8 = (c0 >> 3) + k;
        if (8 * c8 < C) {
            float e[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) e[j] = v[8 * k + j];
            uint4 h;
            h.x = pack_bf2(e[0], e[1]);
            h.y = pack_bf2(e[2], e[3]);
            h.z = pack_bf2(e[4], e[5]);
            h.w = pack_bf2(e[6], e[7]);
            *reinterpret_cast<uint4*>(hi + c8 * (16 * TR) + 16 * r) = h;
            if (lo) {
                uint4 l;
                l.x = pack_bf2(e[0] - bf_hi(e[0]), e[1] - bf_hi(e[1]));
                l.y = pack_bf2(e[2] - bf_hi(e[2]), e[3] - bf_hi(e[3]));
                l.z = pack_bf2(e[4] - bf_hi(e[4]), e[5] - bf_hi(e[5]));
                l.w = pack_bf2(e[6] - bf_hi(e[6]), e[7] - bf_hi(e[7]));
                *reinterpret_cast<uint4*>(lo + c8 * (16 * TR) + 16 * r) = l;
            }
        }
    }
}

// 32 consecutive tensor-memory columns of this warp's lanes
__device__ __forceinline__ void tm_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r0[16], r1[16];
    tc::tmem_ld16(taddr, r0);
    tc::tmem_ld16(taddr + 16, r1);
    tc::tmem_ld_wait();
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        v[j] = __uint_as_float(r0[j]);
        v[16 + j] = __uint_as_float(r1[j]);
    }
}

// logistic sigmoid (the exponential and the reciprocal on the
// special-function unit)
__device__ __forceinline__ float sigm(float u) { return __fdividef(1.f, 1.f + __expf(-u)); }

// Sum of v[0..31] over the warp's lanes by recursive halving: afterwards
// v[0] holds the sum of column `lane`.
__device__ __forceinline__ void warp_colsum32(float (&v)[32], int lane) {
#pragma unroll
    for (int s = 0; s < 5; ++s) {
        const int h = 16 >> s;
        const bool up = lane & h;
#pragma unroll
        for (int j = 0; j < h; ++j) {
            const float send = up ? v[j] : v[j + h];
            const float keep = up ? v[j + h] : v[j];
            v[j] = keep + __shfl_xor_sync(0xffffffffu, send, h);
        }
    }
}

// All threads: bounded wait for the commit with the given parity; the result
// is uniform over the block.
__device__ bool wait_all(uint64_t* bar, uint32_t parity, uint64_t wait_ns, int* d_err, int site) {
    bool ok = true;
    uint64_t deadline = 0;
    for (uint32_t n = 0;; ++n) {
        if (tc::mbar_try_wait(bar, parity, 1000u)) break;
        if ((n & 63u) == 63u) {
            const uint64_t now = tc::globaltimer();
            if (deadline == 0) deadline = now + wait_ns;
            else if (now > deadline) {
                ok = false;
                break;
            }
        }
    }
    tc::fence_after_sync();
    ok = __syncthreads_and(ok);
    if (!ok && threadIdx.x == 0 && atomicCAS(d_err, 0, CS_DEVERR_TIMEOUT) == 0) d_err[1] = site;
    return ok;
}
// After a wait that gave up: one more bounded wait for the MMAs in flight,
// so that the tensor memory is not freed under them.
__device__ void drain(uint64_t* bar, uint32_t parity, uint64_t wait_ns) {
    const uint64_t deadline = tc::globaltimer() + wait_ns;
    while (!tc::mbar_try_wait(bar, parity, 1000u))
        if (tc::globaltimer() > deadline) break;
}

// Generic-proxy shared-memory writes and tensor-memory reads of every thread
// are done before thread 0 issues MMAs.
__device__ __forceinline__ void to_issue() {
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
}

// thread 0: D(128 x N) (+)= [Ah | Al](128 x 2K) [W | W]^T, W a row-layout tile
// of N rows (K-major).
__device__ __forceinline__ void mma_fwd(uint32_t d, const unsigned char* Ah, const unsigned char* Al,
                                        int K, const unsigned char* W, int N) {
    const uint32_t id = tc::idesc(TR, N, 1, 1);
    for (int part = 0; part < 2; ++part) {
        const unsigned char* A = part ? Al : Ah;
        for (int kk = 0; kk < K / 16; ++kk)
            tc::mma_bf16(d, desc_k(A + kk * (32 * TR), TR), desc_k(W + kk * 32 * N, N), id,
                         (part | kk) ? 1u : 0u);
    }
}
// thread 0: P(128 x 64) = D(128 x [hi | lo] of K) W(K x 64), W a row-layout
// tile of K rows read MN-major; D holds hi in columns [0, 64), lo in [64, 128).
__device__ __forceinline__ void mma_prop(uint32_t d, const unsigned char* D, int K,
                                         const unsigned char* W) {
    const uint32_t id = tc::idesc(TR, HID, 1, 1) | B_MN;
    for (int part = 0; part < 2; ++part)
        for (int kk = 0; kk < K / 16; ++kk)
            tc::mma_bf16(d, desc_k(D + (part * 8 + 2 * kk) * (16 * TR), TR),
                         desc_mn(W + kk * 256, K), id, (part | kk) ? 1u : 0u);
}
// thread 0: G(128 x N) (+)= D^T H over the tile's 128 rows: row o' of G is
// output o' of D's hi piece (o' < 64) or of its lo piece (o' - 64).
__device__ __forceinline__ void mma_wgrad(uint32_t g, const unsigned char* D, const unsigned char* H,
                                          int N, bool accumulate) {
    const uint32_t id = tc::idesc(TR, N, 1, 1) | A_MN | B_MN;
    for (int kk = 0; kk < TR / 16; ++kk)
        tc::mma_bf16(g, desc_mn(D + kk * 256, TR), desc_mn(H + kk * 256, TR), id,
                     (accumulate || kk) ? 1u : 0u);
}

// ------------------------------------------------------------------ training
struct TrainLayout {
    uint32_t W1, W2, W3, W4, X, H1, H2, H3, HL, D, F32, BAR, total;
};
__host__ __device__ inline TrainLayout train_layout(int K0, int NOp) {
    TrainLayout L;
    uint32_t o = 0;
    L.W1 = o; o += 2 * HID * K0;
    L.W2 = o; o += 2 * HID * HID;
    L.W3 = o; o += 2 * HID * HID;
    L.W4 = o; o += 2 * NOp * HID;
    L.X = o; o += 2 * TR * K0;
    L.H1 = o; o += 2 * TR * HID;
    L.H2 = o; o += 2 * TR * HID;
    L.H3 = o; o += 2 * TR * HID;
    L.HL = o; o += 2 * TR * HID;
    L.D = o; o += 2 * TR * 2 * HID;
    L.F32 = o; o += 4 * (4 * HID + 2 * 8 * 32 + 8);  // biases, column-sum exchange (x2), loss
    L.BAR = o; o += 32;
    L.total = o;
    return L;
}

struct TrainArgs {
    const unsigned char* image;  // the weight image (bf16 tiles + biases)
    int nin, n;
    const float* X;  // [n_rows][nin] standardised features
    const float* T;  // [n_rows][n] standardised targets
    int n_rows;
    long long start;
    int batch;       // rows of this step: (start + b) mod n_rows, b < batch
    float* part;     // [gridDim.x][PS]: gradient sums, then the loss sum
    int PS;
    int* d_err;
    uint64_t wait_ns;
};

// This thread's half row of the delta into D as hi / lo pieces, and the
// warp's column sums (bias gradient) into ex[warp][lane].
__device__ __forceinline__ void put_delta(float (&dl)[32], int c0, unsigned char* D, float* ex,
                                          int row, int warp, int lane) {
    put_half(dl, c0, HID, D, D + 8 * 16 * TR, row);
    warp_colsum32(dl, lane);
    ex[warp * 32 + lane] = dl[0];
}

__global__ void __launch_bounds__(NTH, 1) mlp_train_kernel(TrainArgs a) {
    extern __shared__ __align__(1024) unsigned char sm[];
    const Dims dm = dims_of(a.nin, a.n);
    const Off of = off_of(a.nin, a.n);
    const TrainLayout L = train_layout(dm.K0, dm.NOp);
    unsigned char *W1 = sm + L.W1, *W2 = sm + L.W2, *W3 = sm + L.W3, *W4 = sm + L.W4;
    unsigned char *Xh = sm + L.X, *H1 = sm + L.H1, *H2 = sm + L.H2, *H3 = sm + L.H3;
    unsigned char *HL = sm + L.HL, *D = sm + L.D;
    float* bias = reinterpret_cast<float*>(sm + L.F32);  // b1 b2 b3 b4, 64 each
    float* ex = bias + 4 * HID;                          // [2][8 warps][32]
    float* lred = ex + 2 * 8 * 32;                       // [8]
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + L.BAR);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + L.BAR + 16);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quarter = warp & 3, c0 = 32 * (warp >> 2);
    const int row = 32 * quarter + lane;  // tile row (tensor-memory lane) of this thread
    uint64_t* lbar = bar + 1;             // weight image arrival
    if (warp == 0) tc::tmem_alloc(tslot, 512);
    if (tid == 0) {
        tc::mbar_init(bar, 1);
        tc::mbar_init(lbar, 1);
        tc::fence_mbar_init();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const bool loaded =
        load_image(a.image, img_wbytes(dm.K0, dm.NOp), W1, bias, lbar, a.wait_ns, a.d_err, 60);
    bool ok = loaded;
    const uint32_t tm = *tslot;
    const uint32_t tl = tm + ((uint32_t)(32 * quarter) << 16) + c0;  // this thread's lanes, columns
    // tensor-memory columns: Z1 0, Z2 64, Z3 128, Z4 192 (then P3 192, P2 128,
    // P1 64); gradients G1 256, G2 320, G3 384, G4 448
    const float inv = 1.f / ((float)a.batch * (float)a.n);
    const int tiles = (a.batch + TR - 1) / TR;
    uint32_t ph = 0;
    float dbias[4] = {0.f, 0.f, 0.f, 0.f};  // thread c < 64: bias gradient column c
    float lsum = 0.f;
    int xb = 0;                             // column-sum exchange buffer
    auto colsum_take = [&](int l) {         // after a block barrier
        if (tid < HID) {
            const float* e = ex + xb * 8 * 32 + (tid >> 5) * 4 * 32 + (tid & 31);
            dbias[l] += (e[0] + e[32]) + (e[64] + e[96]);
        }
        xb ^= 1;
    };
    float v[32], w[32];
    for (int tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x) {
        const bool first = tile == (int)blockIdx.x;
        const int b = tile * TR + row;
        const bool valid = b < a.batch;
        const long long srow = valid ? (a.start + b) % a.n_rows : 0;
        // ---- forward
#pragma unroll
        for (int j = 0; j < 32; ++j)
            v[j] = (valid && c0 + j < a.nin) ? a.X[srow * a.nin + c0 + j] : 0.f;
        put_half(v, c0, dm.K0, Xh, HL, row);
        to_issue();
        if (tid == 0) {
            tc::fence_after_sync();
            mma_fwd(tm + 0, Xh, HL, dm.K0, W1, HID);
            tc::mma_commit(bar);
        }
        if (!(ok = wait_all(bar, ph, a.wait_ns, a.d_err, 61))) break;
        ph ^= 1;
        unsigned char* Hs[3] = {H1, H2, H3};
        const unsigned char* Ws[3] = {W2, W3, W4};
        for (int l = 0; l < 3 && ok; ++l) {
            tm_ld32(tl + 64 * l, v);
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const float u = v[j] + bias[l * HID + c0 + j];
                v[j] = u * sigm(u);
            }
            put_half(v, c0, HID, Hs[l], HL, row);
            to_issue();
            if (tid == 0) {
                tc::fence_after_sync();
                mma_fwd(tm + 64 * (l + 1), Hs[l], HL, HID, Ws[l], l < 2 ? HID : dm.NOp);
                tc::mma_commit(bar);
            }
            ok = wait_all(bar, ph, a.wait_ns, a.d_err, 62 + l);
            if (ok) ph ^= 1;
        }
        if (!ok) break;
        // ---- loss and output delta (columns past NOp are read but not used)
        tm_ld32(tl + 192, v);
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            const int c = c0 + j;
            float dl = 0.f;
            if (valid && c < a.n) {
                dl = v[j] + bias[3 * HID + c] - a.T[srow * a.n + c];
                lsum = fmaf(dl, dl, lsum);
            }
            w[j] = dl * inv;
        }
        put_delta(w, c0, D, ex + xb * 8 * 32, row, warp, lane);
        to_issue();
        colsum_take(3);
        if (tid == 0) {
            tc::fence_after_sync();
            mma_prop(tm + 192, D, dm.NOp, W4);
            mma_wgrad(tm + 448, D, H3, HID, !first);
            tc::mma_commit(bar);
        }
        if (!(ok = wait_all(bar, ph, a.wait_ns, a.d_err, 65))) break;
        ph ^= 1;
        // ---- hidden deltas: D_l = P_l * silu'(Z_l + b_l)
        const unsigned char* Hin[3] = {Xh, H1, H2};
        for (int l = 2; l >= 0 && ok; --l) {
            const int pcol = l == 2 ? 192 : 64 * (l + 1);
            tm_ld32(tl + pcol, v);
            tm_ld32(tl + 64 * l, w);
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const float u = w[j] + bias[l * HID + c0 + j];
                const float sg = sigm(u);
                w[j] = v[j] * (sg * (1.f + u * (1.f - sg)));
            }
            put_delta(w, c0, D, ex + xb * 8 * 32, row, warp, lane);
            to_issue();
            colsum_take(l);
            if (tid == 0) {
                tc::fence_after_sync();
                if (l > 0) mma_prop(tm + 64 * l, D, HID, l == 2 ? W3 : W2);
                mma_wgrad(tm + 256 + 64 * l, D, Hin[l], l == 0 ? dm.K0 : HID, !first);
                tc::mma_commit(bar);
            }
            ok = wait_all(bar, ph, a.wait_ns, a.d_err, 66 + l);
            if (ok) ph ^= 1;
        }
    }
    if (ok) {
        // ---- per-CTA sums to the partials buffer: G rows o' and o' + 64 add up
        float* P = a.part + (size_t)blockIdx.x * a.PS;
        float* S = reinterpret_cast<float*>(D);  // 64 x 65 floats
        for (int l = 0; l < 4; ++l) {
            const int cols = l == 0 ? dm.K0 : HID;
            const int cv = l == 0 ? a.nin : HID, rv = l == 3 ? a.n : HID;
            const int woff = l == 0 ? of.W1 : l == 1 ? of.W2 : l == 2 ? of.W3 : of.W4;
            const int boff = l == 0 ? of.b1 : l == 1 ? of.b2 : l == 2 ? of.b3 : of.b4;
            if (c0 < cols) tm_ld32(tl + 256 + 64 * l, v);
            __syncthreads();
            if (row >= HID && c0 < cols) {
#pragma unroll
                for (int j = 0; j < 32; ++j) S[(row - HID) * 65 + c0 + j] = v[j];
            }
            __syncthreads();
            if (row < HID && c0 < cols) {
#pragma unroll
                for (int j = 0; j < 32; ++j) S[row * 65 + c0 + j] += v[j];
            }
            __syncthreads();
            for (int i = tid; i < rv * cv; i += NTH) P[woff + i] = S[(i / cv) * 65 + i % cv];
            if (tid < rv) P[boff + tid] = dbias[l];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
        if (lane == 0) lred[warp] = lsum;
        __syncthreads();
        if (tid == 0) {
            float t = 0.f;
            for (int k = 0; k < NTH / 32; ++k) t += lred[k];
            P[of.np] = 0.5f * inv * t;
        }
    } else {
        drain(loaded ? bar : lbar, loaded ? ph : 0u, a.wait_ns);  // copies or MMAs in flight
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tm, 512);
    }
}

// g_i = sum over the CTAs of the partials (fixed order); then, when m is
// given, bias-corrected Adam on the fp32 masters. Index np: the loss.
// A block covers 32 consecutive indices (one per lane, coalesced) with its 8
// warps taking every 8th CTA, so each thread's loads are independent; the
// warps' sums are added in warp order.
constexpr int RED_W = 8;
__global__ void __launch_bounds__(32 * RED_W) reduce_adam_kernel(
    const float* __restrict__ part, int G, int PS, int np, float* __restrict__ p,
    float* __restrict__ g_out, float* __restrict__ m, float* __restrict__ v, float lr, float b1,
    float b2, float eps, float c1, float c2, float* __restrict__ loss, unsigned char* image,
    int nin, int n) {
    __shared__ float acc[RED_W][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int i = blockIdx.x * 32 + lane;
    float s = 0.f;
    if (i <= np) {
#pragma unroll 4
        for (int c = w; c < G; c += RED_W) s += part[(size_t)c * PS + i];
    }
    acc[w][lane] = s;
    __syncthreads();
    if (w != 0 || i > np) return;
    float g = 0.f;
#pragma unroll
    for (int k = 0; k < RED_W; ++k) g += acc[k][lane];
    if (i == np) {
        if (loss) *loss = g;
        return;
    }
    if (g_out) g_out[i] = g;
    if (m) {
        const float mi = b1 * m[i] + (1.f - b1) * g;
        const float vi = b2 * v[i] + (1.f - b2) * g * g;
        m[i] = mi;
        v[i] = vi;
        const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        p[i] = pi;
        if (image) img_store(image, off_of(nin, n), dims_of(nin, n), i, pi);
    }
}

// the image of the given parameters (zero-filled beforehand)
__global__ void pack_kernel(const float* __restrict__ p, int nin, int n, unsigned char* image) {
    const Off of = off_of(nin, n);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < of.np) img_store(image, of, dims_of(nin, n), i, p[i]);
}

// ------------------------------------------------------------------ features
struct FeatSrc {
    const float* img;
    const float* lead16;
    const int32_t* dist2;  // [n][P] squared scribble distances (feature set 1)
    int H, W, n, set;
    float d_min;
};

// Raw feature c of pixel q = y W + x: [R, G, B, x/W, y/H, a_1..a_16], then
// for feature set 1 log max(d_i, d_min) for every label i and sin, cos of
// 2^f pi x/W and of 2^f pi y/H for f = 0..5 (the argument reduced exactly:
// 2^f x mod 2W). Images hold fewer than 2^31 pixels.
__device__ __forceinline__ float pixel_feature(const FeatSrc& s, int q, int x, int y, int c) {
    if (c < 3) return s.img[(size_t)q * 3 + c];
    if (c == 3) return (float)x / (float)s.W;
    if (c == 4) return (float)y / (float)s.H;
    if (c < 21) return s.lead16[(size_t)q * 16 + (c - 5)];
    if (s.set == 0) return 0.f;
    c -= 21;
    if (c < s.n)
        return logf(fmaxf(sqrtf((float)s.dist2[(size_t)c * s.H * s.W + q]), s.d_min));
    c -= s.n;
    if (c >= 24) return 0.f;
    const int f = c >> 2, kind = c & 3;
    const int w = kind < 2 ? s.W : s.H;
    const int m = (int)(((long long)(kind < 2 ? x : y) << f) % (2LL * w));
    const float t = (float)m / (float)w;
    return (kind & 1) ? cospif(t) : sinpif(t);
}

// ------------------------------------------------------------------ forward
enum { SRC_ROWS = 0, SRC_EVAL = 1 };

struct FwdArgs {
    const unsigned char* image;  // the weight image (bf16 tiles + biases)
    int nin, n;
    const float* X;  // SRC_ROWS: [rows][nin] standardised
    int rows;
    float* Z;        // SRC_ROWS: [rows][n]
    // SRC_EVAL
    FeatSrc fs;
    const float* stats;  // mu_x[nin] sd_x[nin] mu_t[n] sd_t[n]
    const float* eta;
    const int32_t* label_off;
    const uint32_t* bitmask;
    const uint32_t* rep;
    int Wk, mode, rule;
    float alpha, kappa_beta, sigma_c2, margin, eps;
    bool rho_var;
    float* neglog;
    float* post;
    int32_t* fb_list;
    int* fb_count;
    int* d_err;
    uint64_t wait_ns;
};

struct FwdLayout {
    uint32_t W1, W2, W3, W4, HH, HL, F32, BAR, total;
};
__host__ __device__ inline FwdLayout fwd_layout(int K0, int NOp) {
    FwdLayout L;
    uint32_t o = 0;
    L.W1 = o; o += 2 * HID * K0;
    L.W2 = o; o += 2 * HID * HID;
    L.W3 = o; o += 2 * HID * HID;
    L.W4 = o; o += 2 * NOp * HID;
    L.HH = o; o += 2 * TR * HID;
    L.HL = o; o += 2 * TR * HID;
    L.F32 = o; o += 4 * (4 * HID + 4 * 64);  // biases; mu_x sd_x mu_t sd_t
    L.BAR = o; o += 32;
    L.total = o;
    return L;
}

// Surrogate post-processing of one pixel (see the file header).
__device__ void eval_pixel(const FwdArgs& a, long long q, float (&z)[64], const float* mu_t,
                           const float* sd_t, float gap_min) {
    const int n = a.n;
    const long long P = (long long)a.fs.H * a.fs.W;
    const float log_col_norm = 1.5f * logf(6.283185307179586f * a.sigma_c2);
    uint32_t bx[8];
    for (int w = 0; w < 8; ++w)
        bx[w] = (a.mode == CS_MODE_FACTORISED && w < a.Wk) ? a.bitmask[q * a.Wk + w] : 0u;
    float tmax = -INFINITY;
    float tex[64];  // factorised mode: the texture exponents -h_j / beta_j
    for (int j = 0; j < n; ++j) {
        const float rho = a.alpha * fmaxf(sqrtf((float)a.fs.dist2[(size_t)j * P + q]), a.fs.d_min);
        const float T = z[j] * sd_t[j] + mu_t[j];
        z[j] = T - logf((float)(a.label_off[j + 1] - a.label_off[j])) -
               logf(6.283185307179586f * (a.rho_var ? rho : rho * rho)) - log_col_norm;
        if (a.mode == CS_MODE_FACTORISED) {
            int h = 0;
            for (int w = 0; w < a.Wk; ++w) h += __popc(bx[w & 7] ^ a.rep[j * a.Wk + w]);
            tex[j] = -(float)h / (a.kappa_beta * rho);
            tmax = fmaxf(tmax, tex[j]);
        }
    }
    if (a.mode == CS_MODE_FACTORISED) {
        float ts = 0.f;
        for (int j = 0; j < n; ++j) ts += expf(tex[j] - tmax);
        const float tl = tmax + logf(ts);
        for (int j = 0; j < n; ++j) z[j] += tex[j] - tl;
    }
    float m1 = -INFINITY, m2 = -INFINITY;
    for (int j = 0; j < n; ++j) {
        if (z[j] > m1) {
            m2 = m1;
            m1 = z[j];
        } else if (z[j] > m2) {
            m2 = z[j];
        }
    }
    float ls = 0.f;
    for (int j = 0; j < n; ++j) ls += expf(z[j] - m1);
    const float lse = m1 + logf(ls);
    const float p1 = expf(m1 - lse), p2 = n > 1 ? expf(m2 - lse) : 0.f;
    const bool fb = a.rule != CS_FALLBACK_NONE &&
                    ((p1 - p2 < a.margin) ||
                     (a.rule == CS_FALLBACK_GUARANTEED && n > 1 && m1 - m2 < gap_min));
    if (fb) {
        const int idx = atomicAdd(a.fb_count, 1);
        if (idx < P) a.fb_list[idx] = (int32_t)q;
        return;
    }
    for (int j = 0; j < n; ++j) {
        a.neglog[(size_t)j * P + q] = -z[j];
        if (a.post) a.post[(size_t)j * P + q] = expf(z[j] - lse);
    }
}

template <int SRC>
__global__ void __launch_bounds__(NTH, 2) mlp_fwd_kernel(FwdArgs a) {
    extern __shared__ __align__(1024) unsigned char sm[];
    const Dims dm = dims_of(a.nin, a.n);
    const FwdLayout L = fwd_layout(dm.K0, dm.NOp);
    unsigned char *W1 = sm + L.W1, *W2 = sm + L.W2, *W3 = sm + L.W3, *W4 = sm + L.W4;
    unsigned char *HH = sm + L.HH, *HL = sm + L.HL;
    float* ZS = reinterpret_cast<float*>(HH);  // [128][33]: upper output half (HH and HL)
    float* bias = reinterpret_cast<float*>(sm + L.F32);
    float* mu_x = bias + 4 * HID;
    float* sd_x = mu_x + 64;
    float* mu_t = sd_x + 64;
    float* sd_t = mu_t + 64;
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + L.BAR);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + L.BAR + 16);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quarter = warp & 3, c0 = 32 * (warp >> 2);
    const int row = 32 * quarter + lane;
    if (SRC == SRC_EVAL)
        for (int i = tid; i < 64; i += NTH) {
            mu_x[i] = i < a.nin ? a.stats[i] : 0.f;
            sd_x[i] = i < a.nin ? a.stats[a.nin + i] : 1.f;
            mu_t[i] = i < a.n ? a.stats[2 * a.nin + i] : 0.f;
            sd_t[i] = i < a.n ? a.stats[2 * a.nin + a.n + i] : 1.f;
        }
    uint64_t* lbar = bar + 1;  // weight image arrival
    if (warp == 0) tc::tmem_alloc(tslot, 64);
    if (tid == 0) {
        tc::mbar_init(bar, 1);
        tc::mbar_init(lbar, 1);
        tc::fence_mbar_init();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const bool loaded =
        load_image(a.image, img_wbytes(dm.K0, dm.NOp), W1, bias, lbar, a.wait_ns, a.d_err, 70);
    bool ok = loaded;
    const uint32_t tm = *tslot;
    const uint32_t tl = tm + ((uint32_t)(32 * quarter) << 16) + c0;
    const long long total = SRC == SRC_ROWS ? (long long)a.rows : (long long)a.fs.H * a.fs.W;
    const long long tiles = (total + TR - 1) / TR;
    float gap_min = 0.f;
    if (SRC == SRC_EVAL)  // a gap g keeps the max probability error <= eps when
                          // every logit is within eta of the truth:
                          // (n - 1) exp(-(g - 2 eta)) <= eps
        gap_min = 2.2f * (*a.eta) + logf(fmaxf((float)(a.n - 1), 1.f) / a.eps);
    uint32_t ph = 0;
    float v[32];
    for (long long tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x) {
        const long long r = tile * TR + row;
        const bool valid = r < total;
        if (SRC == SRC_ROWS) {
#pragma unroll
            for (int j = 0; j < 32; ++j)
                v[j] = (valid && c0 + j < a.nin) ? a.X[r * a.nin + c0 + j] : 0.f;
        } else {
            const int q = valid ? (int)r : 0, y = q / a.fs.W, x = q - y * a.fs.W;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const int c = c0 + j;
                v[j] = (valid && c < a.nin) ? (pixel_feature(a.fs, q, x, y, c) - mu_x[c]) / sd_x[c]
                                            : 0.f;
            }
        }
        put_half(v, c0, dm.K0, HH, HL, row);
        for (int l = 0; l < 4; ++l) {
            to_issue();
            if (tid == 0) {
                tc::fence_after_sync();
                mma_fwd(tm, HH, HL, l == 0 ? dm.K0 : HID, l == 0 ? W1 : l == 1 ? W2 : l == 2 ? W3 : W4,
                        l < 3 ? HID : dm.NOp);
                tc::mma_commit(bar);
            }
            if (!(ok = wait_all(bar, ph, a.wait_ns, a.d_err, 71 + l))) break;
            ph ^= 1;
            tm_ld32(tl, v);  // the last layer: columns past NOp are read but not used
            if (l < 3) {
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const float u = v[j] + bias[l * HID + c0 + j];
                    v[j] = u * sigm(u);
                }
                put_half(v, c0, HID, HH, HL, row);
            }
        }
        if (!ok) break;
        tc::fence_before_sync();  // the next tile's MMAs overwrite these columns
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] += bias[3 * HID + c0 + j];
        if (SRC == SRC_ROWS) {
            if (valid) {
#pragma unroll
                for (int j = 0; j < 32; ++j)
                    if (c0 + j < a.n) a.Z[r * a.n + c0 + j] = v[j];
            }
        } else {
            // one thread per pixel takes the labels' post-processing; for more
            // than 32 labels the upper half comes through shared memory
            float z[64];
#pragma unroll
            for (int j = 0; j < 32; ++j) z[j] = v[j];
            if (a.n > 32) {
                if (c0) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) ZS[row * 33 + j] = v[j];
                }
                __syncthreads();
                if (!c0) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) z[32 + j] = ZS[row * 33 + j];
                }
                __syncthreads();  // ZS is the next tile's operand space
            }
            if (!c0 && valid) eval_pixel(a, r, z, mu_t, sd_t, gap_min);
        }
    }
    if (!ok) drain(loaded ? bar : lbar, loaded ? ph : 0u, a.wait_ns);  // copies or MMAs in flight
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tm, 64);
    }
}

// ------------------------------------------------------------------ data preparation
__global__ void features_kernel(FeatSrc s, int nin, const int32_t* __restrict__ list, int rows,
                                float* __restrict__ X) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)rows * nin) return;
    const long long r = i / nin;
    const int q = list[r], y = q / s.W, x = q - y * s.W;
    X[i] = pixel_feature(s, q, x, y, (int)(i % nin));
}

// one block per column: mean and standard deviation over the first n_rows
// rows, in double, deterministic tree reduction. Columns 0..nin-1 come from
// X (row-major, stride nin); nin..nin+n-1 from T (label-major, stride cap).
__global__ void stats_kernel(const float* __restrict__ X, int nin, const float* __restrict__ T,
                             int n, int cap, int n_rows, float* __restrict__ stats) {
    __shared__ double red[2][256];
    const int c = blockIdx.x;
    double s = 0.0, s2 = 0.0;
    for (int r = threadIdx.x; r < n_rows; r += blockDim.x) {
        const double v = c < nin ? (double)X[(size_t)r * nin + c] : (double)T[(size_t)(c - nin) * cap + r];
        s += v;
        s2 += v * v;
    }
    red[0][threadIdx.x] = s;
    red[1][threadIdx.x] = s2;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            red[0][threadIdx.x] += red[0][threadIdx.x + w];
            red[1][threadIdx.x] += red[1][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double mu = red[0][0] / n_rows;
        const double var = red[1][0] / n_rows - mu * mu;
        const double sd = var > 1e-12 ? sqrt(var) : 1.0;
        // layout: mu_x[nin] sd_x[nin] mu_t[n] sd_t[n]
        if (c < nin) {
            stats[c] = (float)mu;
            stats[nin + c] = (float)sd;
        } else {
            stats[2 * nin + (c - nin)] = (float)mu;
            stats[2 * nin + n + (c - nin)] = (float)sd;
        }
    }
}

// X <- (X - mu_x) / sd_x in place; Ts[r][j] = (T[j][r] - mu_t,j) / sd_t,j
__global__ void standardize_kernel(float* __restrict__ X, int nin, const float* __restrict__ T,
                                   int n, int cap, int rows, const float* __restrict__ stats,
                                   float* __restrict__ Ts) {
    const long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (r >= rows) return;
    for (int c = 0; c < nin; ++c) X[r * nin + c] = (X[r * nin + c] - stats[c]) / stats[nin + c];
    for (int j = 0; j < n; ++j)
        Ts[r * n + j] = (T[(size_t)j * cap + r] - stats[2 * nin + j]) / stats[2 * nin + n + j];
}

__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

// Glorot-uniform weights from a counter-based generator, zero biases, zero
// optimiser state.
__global__ void init_params_kernel(float* __restrict__ p, float* __restrict__ m,
                                   float* __restrict__ v, int nin, int n, uint64_t seed) {
    const Off o = off_of(nin, n);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= o.np) return;
    float w = 0.f;
    int fan_in = 0, fan_out = 0;
    if (i < o.b1) { fan_in = nin; fan_out = HID; }
    else if (i >= o.W2 && i < o.b2) { fan_in = HID; fan_out = HID; }
    else if (i >= o.W3 && i < o.b3) { fan_in = HID; fan_out = HID; }
    else if (i >= o.W4 && i < o.b4) { fan_in = HID; fan_out = n; }
    if (fan_in) {
        const double u = (double)(splitmix64(seed ^ (0xA5A5A5A5ull + (uint64_t)i)) >> 11) * 0x1.0p-53;
        const double lim = sqrt(6.0 / (fan_in + fan_out));
        w = (float)((2.0 * u - 1.0) * lim);
    }
    p[i] = w;
    m[i] = 0.f;
    v[i] = 0.f;
}

// largest |z - t| * sd_t over rows and labels (a positive float: max via int bits)
__global__ void calib_kernel(const float* __restrict__ Z, const float* __restrict__ Ts, int nin,
                             int n, int rows, const float* __restrict__ stats,
                             float* __restrict__ eta) {
    const long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (r >= rows) return;
    float mx = 0.f;
    for (int j = 0; j < n; ++j)
        mx = fmaxf(mx, fabsf(Z[r * n + j] - Ts[r * n + j]) * stats[2 * nin + n + j]);
    atomicMax(reinterpret_cast<int*>(eta), __float_as_int(mx));
}

cudaError_t set_smem(const void* fn, size_t bytes) {
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

int mlp_param_count(int nin, int n) { return off_of(nin, n).np; }

size_t mlp_image_bytes(int nin, int n) {
    const Dims dm = dims_of(nin, n);
    return img_bytes(dm.K0, dm.NOp);
}

cudaError_t launch_mlp_pack(const float* params, int nin, int n, unsigned char* image,
                            cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(image, 0, mlp_image_bytes(nin, n), st);
    if (e != cudaSuccess) return e;
    const int np = mlp_param_count(nin, n);
    pack_kernel<<<(np + 255) / 256, 256, 0, st>>>(params, nin, n, image);
    return cudaGetLastError();
}

int mlp_train_ctas(int batch, int n_sm) {
    const int tiles = (batch + TR - 1) / TR;
    return tiles < n_sm ? tiles : n_sm;
}
int mlp_part_stride(int nin, int n) { return (off_of(nin, n).np + 1 + 3) & ~3; }

cudaError_t launch_mlp_train(const unsigned char* image, int nin, int n, const float* X, const float* T,
                             int n_rows, long long start, int batch, float* part, int G,
                             int* d_err, uint64_t wait_ns, cudaStream_t st) {
    const Dims dm = dims_of(nin, n);
    const size_t smem = train_layout(dm.K0, dm.NOp).total;
    cudaError_t e = set_smem((const void*)mlp_train_kernel, smem);
    if (e != cudaSuccess) return e;
    TrainArgs a{image, nin, n, X, T, n_rows, start, batch, part, mlp_part_stride(nin, n), d_err,
                wait_ns ? wait_ns : MLP_WAIT_NS};
    mlp_train_kernel<<<G, NTH, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_reduce_adam(const float* part, int G, int nin, int n, float* p, float* g_out,
                               float* m, float* v, float lr, int t, float* loss,
                               unsigned char* image, cudaStream_t st) {
    const int np = mlp_param_count(nin, n);
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
    reduce_adam_kernel<<<(np + 1 + 31) / 32, 32 * RED_W, 0, st>>>(part, G, mlp_part_stride(nin, n), np,
                                                                  p, g_out, m, v, lr, b1, b2, 1e-8f,
                                                                  c1, c2, loss, image, nin, n);
    return cudaGetLastError();
}

static int fwd_grid(long long total, int n_sm) {
    const long long tiles = (total + TR - 1) / TR;
    const long long cap = 2LL * n_sm;  // two CTAs per SM (registers)
    return (int)(tiles < cap ? tiles : cap);
}

cudaError_t launch_mlp_forward(const unsigned char* image, int nin, int n, const float* X, int rows,
                               float* Z, int n_sm, int* d_err, uint64_t wait_ns, cudaStream_t st) {
    const Dims dm = dims_of(nin, n);
    const size_t smem = fwd_layout(dm.K0, dm.NOp).total;
    cudaError_t e = set_smem((const void*)mlp_fwd_kernel<SRC_ROWS>, smem);
    if (e != cudaSuccess) return e;
    FwdArgs a{};
    a.image = image;
    a.nin = nin;
    a.n = n;
    a.X = X;
    a.rows = rows;
    a.Z = Z;
    a.d_err = d_err;
    a.wait_ns = wait_ns ? wait_ns : MLP_WAIT_NS;
    mlp_fwd_kernel<SRC_ROWS><<<fwd_grid(rows, n_sm), NTH, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_surrogate_eval(const SurrogateEvalArgs& s, cudaStream_t st) {
    const Dims dm = dims_of(s.nin, s.n);
    const size_t smem = fwd_layout(dm.K0, dm.NOp).total;
    cudaError_t e = set_smem((const void*)mlp_fwd_kernel<SRC_EVAL>, smem);
    if (e != cudaSuccess) return e;
    FwdArgs a{};
    a.image = s.image;
    a.nin = s.nin;
    a.n = s.n;
    a.fs = FeatSrc{s.img, s.lead16, s.dist2, s.H, s.W, s.n, s.feature_set, s.d_min};
    a.stats = s.stats;
    a.eta = s.eta;
    a.label_off = s.label_off;
    a.bitmask = s.bitmask;
    a.rep = s.rep;
    a.Wk = s.Wk;
    a.mode = s.mode;
    a.rule = s.rule;
    a.alpha = s.alpha;
    a.kappa_beta = s.kappa_beta;
    a.sigma_c2 = s.sigma_c2;
    a.margin = s.margin;
    a.eps = s.eps;
    a.rho_var = s.rho_var;
    a.neglog = s.neglog;
    a.post = s.post;
    a.fb_list = s.fb_list;
    a.fb_count = s.fb_count;
    a.d_err = s.d_err;
    a.wait_ns = s.wait_ns ? s.wait_ns : MLP_WAIT_NS;
    mlp_fwd_kernel<SRC_EVAL><<<fwd_grid((long long)s.H * s.W, s.n_sm), NTH, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_features(const float* img, const float* lead16, const int32_t* dist2, int H,
                            int W, int n, int feature_set, float d_min, int nin,
                            const int32_t* list, int rows, float* X, cudaStream_t st) {
    const long long total = (long long)rows * nin;
    FeatSrc s{img, lead16, dist2, H, W, n, feature_set, d_min};
    features_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(s, nin, list, rows, X);
    return cudaGetLastError();
}

cudaError_t launch_stats(const float* X, int nin, const float* T, int n, int cap, int n_rows,
                         float* stats, cudaStream_t st) {
    stats_kernel<<<nin + n, 256, 0, st>>>(X, nin, T, n, cap, n_rows, stats);
    return cudaGetLastError();
}

cudaError_t launch_standardize(float* X, int nin, const float* T, int n, int cap, int rows,
                               const float* stats, float* Ts, cudaStream_t st) {
    standardize_kernel<<<(rows + 127) / 128, 128, 0, st>>>(X, nin, T, n, cap, rows, stats, Ts);
    return cudaGetLastError();
}

cudaError_t launch_init_params(float* p, float* m, float* v, int nin, int n, uint64_t seed,
                               cudaStream_t st) {
    const int np = mlp_param_count(nin, n);
    init_params_kernel<<<(np + 255) / 256, 256, 0, st>>>(p, m, v, nin, n, seed);
    return cudaGetLastError();
}

cudaError_t launch_calib(const float* Z, const float* Ts, int nin, int n, int rows,
                         const float* stats, float* eta, cudaStream_t st) {
    calib_kernel<<<(rows + 127) / 128, 128, 0, st>>>(Z, Ts, nin, n, rows, stats, eta);
    return cudaGetLastError();
}
