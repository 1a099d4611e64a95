// Exact squared distance from every pixel to the nearest scribble sample of
// each label (Sec. 3.1: rho_i(x) = alpha |x - x_v|, x_v the closest scribble
// location of label i).
//
// Separable exact transform in integers:
//   1. seed bitmaps: one bit per pixel and label;
//   2. row pass (one warp per label and row): horizontal distance h to the
//      nearest seed in the same row, from bit scans of the bitmap words;
//   3. column pass (2, 4 or 8 builder threads per label and column, one per
//      row segment, and eight readers): lower envelopes of the parabolas
//      (y - q)^2 + h(q)^2 over each segment's rows q with finite h, each
//      built in one sweep and read back by row ranges; intersection
//      abscissae are compared as exact rationals with 64-bit cross products,
//      so the result equals the brute-force minimum bit for bit. For images
//      with few columns and rows (labels x width < 16384, height <= 64) an
//      outward scan per pixel with early exit gives the same minimum with
//      far more parallelism.
// The sample gather builds SoA tables of every sample (location, colour,
// co-support bitmask and its popcount) and, for the factorised form, the
// majority co-support of each label (Eq. tex-rep: bit set iff 2 * count >= m).
#include <algorithm>
#include <cstdint>
#include <type_traits>

#include "internal.h"

namespace {

constexpr int32_t INF = 0x7FFFFFFF;

__device__ __forceinline__ int label_of(const int32_t* __restrict__ off, int n_labels, int s) {
    int lo = 0, hi = n_labels - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= s)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// Seed bitmap: bit (x & 31) of word [i][y][x >> 5] is set when (y, x) is a
// sample of label i.
__global__ void seed_kernel(const int32_t* __restrict__ off, int n_labels,
                            const int32_t* __restrict__ sample_pix, int n_samples, int H, int W,
                            uint32_t* __restrict__ bm, int* __restrict__ d_err) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_samples) return;
    const int pix = sample_pix[s];
    if (pix < 0 || pix >= H * W) {  // reject out-of-image sample indices, never write them
        if (atomicCAS(d_err, 0, CS_DEVERR_BAD_SAMPLE) == 0) d_err[1] = s;
        return;
    }
    const int i = label_of(off, n_labels, s);
    const int y = pix / W, x = pix % W, Wb = (W + 31) >> 5;
    atomicOr(bm + ((size_t)i * H + y) * Wb + (x >> 5), 1u << (x & 31));
}

// Pass 1 (one warp per label and row): horizontal distance to the nearest
// seed of the same row (INF if the row has none), from the seed bitmap with
// ballot-free bit scans; a forward sweep finds the last seed at or left of
// each pixel, a backward sweep the next seed at or right of it.
__global__ void rows_binary_kernel(int H, int W, int n_labels, const uint32_t* __restrict__ bm,
                                   int32_t* __restrict__ h) {
    const long long row = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= (long long)n_labels * H) return;
    const int Wb = (W + 31) >> 5;
    const uint32_t* b = bm + (size_t)row * Wb;
    int32_t* out = h + (size_t)row * W;
    int carry = -1;  // last seed column seen so far
    for (int c = 0; c < Wb; ++c) {
        const uint32_t word = b[c];
        const uint32_t le = word & (lane == 31 ? 0xFFFFFFFFu : ((2u << lane) - 1u));
        const int last = le ? 32 * c + 31 - __clz(le) : carry;
        const int x = 32 * c + lane;
        if (x < W) out[x] = last < 0 ? INF : x - last;
        if (word) carry = 32 * c + 31 - __clz(word);
    }
    carry = -1;  // next seed column seen so far (from the right)
    for (int c = Wb - 1; c >= 0; --c) {
        const uint32_t word = b[c];
        const uint32_t ge = word & (0xFFFFFFFFu << lane);
        const int next = ge ? 32 * c + __ffs(ge) - 1 : carry;
        const int x = 32 * c + lane;
        if (x < W && next >= 0 && next - x < out[x]) out[x] = next - x;
        if (word) carry = 32 * c + __ffs(word) - 1;
    }
}

// Column pass, split: in each block of 32 columns S warps build the lower
// envelopes of every column, warp b over the rows of segment b (one thread
// per column and segment; one sweep over the segment's rows with finite h: a
// row's parabola (y - q)^2 + h(q)^2 replaces the stack top while it lies
// below it from the top's breakpoint on, compared exactly with 64-bit cross
// products); then all NSEG warps read them back, warp s for the rows
// [s H / NSEG, (s + 1) H / NSEG): each thread finds the segment of its first
// row in each of the S envelopes by binary search over the breakpoints (the
// same exact comparison, monotone in the segment index), walks on, and keeps
// the smallest of the S values, the minimum over all rows. More segments
// shorten the sequential sweeps at the cost of more envelopes per read.
constexpr int NSEG = 8;  // reader warps per block (and the most segments)


__device__ __forceinline__ int env_build(const int32_t* __restrict__ col, int W, int q_lo, int q_hi,
                                         int32_t* v, int32_t* F, long long stride) {
    int kk = -1;
    constexpr int PF = 16;  // rows of h fetched ahead (independent loads)
    for (int q0 = q_lo; q0 < q_hi; q0 += PF) {
        int32_t hv[PF];
#pragma unroll
        for (int u = 0; u < PF; ++u) hv[u] = q0 + u < q_hi ? col[(size_t)(q0 + u) * W] : INF;
#pragma unroll
        for (int u = 0; u < PF; ++u) {
            const int q = q0 + u;
            const int32_t hq = hv[u];
            if (hq == INF) continue;
            const int32_t Fq = hq * hq + q * q;
            while (kk > 0) {
                const int vk = v[kk * stride], vp = v[(kk - 1) * stride];
                const int32_t Fv = F[kk * stride], Fp = F[(kk - 1) * stride];
                if ((long long)(Fq - Fv) * (vk - vp) <= (long long)(Fv - Fp) * (q - vk))
                    --kk;
                else
                    break;
            }
            ++kk;
            v[kk * stride] = q;
            F[kk * stride] = Fq;
        }
    }
    return kk;
}

// Reader state on one envelope: current segment j (vertex vj, value Fj).
struct EnvCursor {
    int j, kk, vj;
    int32_t Fj;
};
__device__ __forceinline__ EnvCursor env_seek(const int32_t* v, const int32_t* F,
                                              long long stride, int kk, int y0) {
    int lo = 0, hi = kk;
    while (lo < hi) {  // first segment whose right breakpoint is not left of y0
        const int mid = (lo + hi) >> 1;
        const int vm = v[mid * stride], vn = v[(mid + 1) * stride];
        const int32_t Fm = F[mid * stride], Fn = F[(mid + 1) * stride];
        if ((long long)(Fn - Fm) < 2ll * y0 * (vn - vm)) lo = mid + 1;  // z(v_mid, v_mid+1) < y0
        else hi = mid;
    }
    return {lo, kk, v[lo * stride], F[lo * stride]};
}
__device__ __forceinline__ int32_t env_value(EnvCursor& c, const int32_t* v, const int32_t* F,
                                             long long stride, int y) {
    while (c.j < c.kk) {
        const int vn = v[(c.j + 1) * stride];
        const int32_t Fn = F[(c.j + 1) * stride];
        if ((long long)(Fn - c.Fj) < 2ll * y * (vn - c.vj)) {  // z(vj, vn) < y
            ++c.j;
            c.vj = vn;
            c.Fj = Fn;
        } else {
            break;
        }
    }
    return (y - c.vj) * (y - c.vj) + (c.Fj - c.vj * c.vj);
}

template <bool SHARED, int S>
__global__ void __launch_bounds__(32 * NSEG) cols_envelope_split_kernel(
    int H, int W, int n_labels, const int32_t* __restrict__ h, int32_t* __restrict__ gv,
    int32_t* __restrict__ gF, int32_t* __restrict__ dist2) {
    static_assert(S >= 1 && S <= NSEG, "segments");
    extern __shared__ int32_t smem[];
    __shared__ int s_kk[S][32];
    const long long ncol = (long long)n_labels * W;
    const int c = threadIdx.x & 31, seg = threadIdx.x >> 5;
    const long long col_id = blockIdx.x * 32ll + c;
    const bool valid = col_id < ncol;
    const int i = valid ? (int)(col_id / W) : 0, x = valid ? (int)(col_id % W) : 0;
    const int HS = (H + S - 1) / S;  // rows (and stack entries) per segment
    int32_t *v, *F;
    long long stride;
    if (SHARED) {
        v = smem + c;
        F = smem + (size_t)S * HS * 32 + c;
        stride = 32;
    } else {
        v = gv + col_id;
        F = gF + col_id;
        stride = ncol;
    }
    const int32_t* col = h + (size_t)i * H * W + x;
    if (seg < S && valid) {
        const int q_lo = seg * HS, q_hi = min(H, q_lo + HS);
        s_kk[seg][c] = q_lo < q_hi ? env_build(col, W, q_lo, q_hi, v + (size_t)seg * HS * stride,
                                               F + (size_t)seg * HS * stride, stride)
                                   : -1;
    }
    __syncthreads();  // envelopes complete (shared or global) for the whole block
    if (!valid) return;
    int32_t* out = dist2 + (size_t)i * H * W + x;
    const int y0 = (int)((long long)H * seg / NSEG), y1 = (int)((long long)H * (seg + 1) / NSEG);
    EnvCursor cur[S];
    int kk[S];
#pragma unroll
    for (int b = 0; b < S; ++b) {
        kk[b] = s_kk[b][c];
        if (kk[b] >= 0)
            cur[b] = env_seek(v + (size_t)b * HS * stride, F + (size_t)b * HS * stride, stride,
                              kk[b], y0);
    }
    for (int y = y0; y < y1; ++y) {
        int32_t d = INF;  // INF when the label has no valid seed (a bad sample index)
#pragma unroll
        for (int b = 0; b < S; ++b)
            if (kk[b] >= 0)
                d = min(d, env_value(cur[b], v + (size_t)b * HS * stride,
                                     F + (size_t)b * HS * stride, stride, y));
        out[(size_t)y * W] = d;
    }
}

// Column pass for small images (one thread per label and pixel, x fastest):
// D(y) = min over rows q of h(q)^2 + (y - q)^2, scanning q outwards from y
// and stopping once (y - q)^2 alone reaches the best value found, which no
// farther row can beat. Exact (integer arithmetic); O(min(H, sqrt(D))) per
// pixel, so it is chosen only for short images whose envelope pass has too
// few columns to fill the GPU.
__global__ void cols_scan_kernel(int H, int W, int n_labels, const int32_t* __restrict__ h,
                                 int32_t* __restrict__ dist2) {
    const long long P = (long long)H * W;
    const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (tid >= P * n_labels) return;
    const int i = (int)(tid / P);
    const int rem = (int)(tid % P), y = rem / W, x = rem % W;
    const int32_t* col = h + (size_t)i * P + x;
    const int32_t h0 = col[(size_t)y * W];
    int32_t D = h0 == INF ? INF : h0 * h0;
    for (int d = 1; d < H; ++d) {
        const int32_t d2 = d * d;
        if (d2 >= D) break;
        const bool up = y >= d, dn = y + d < H;
        if (!up && !dn) break;
        if (up) {
            const int32_t a = col[(size_t)(y - d) * W];
            if (a != INF) D = min(D, a * a + d2);
        }
        if (dn) {
            const int32_t b = col[(size_t)(y + d) * W];
            if (b != INF) D = min(D, b * b + d2);
        }
    }
    dist2[(size_t)i * P + rem] = D;
}

__global__ void gather_kernel(const float* __restrict__ img, int W, long long P,
                              const uint32_t* __restrict__ bitmask, int Wk,
                              const int32_t* __restrict__ sample_pix, int n_samples,
                              SampleTables t) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_samples) return;
    int pix = sample_pix[s];
    if (pix < 0 || pix >= P) pix = 0;  // reported by seed_kernel; keep the tables finite
    t.sx[s] = (float)(pix % W);
    t.sy[s] = (float)(pix / W);
    t.sr[s] = img[(size_t)pix * 3 + 0];
    t.sg[s] = img[(size_t)pix * 3 + 1];
    t.sb[s] = img[(size_t)pix * 3 + 2];
    int pc = 0;
    for (int w = 0; w < Wk; ++w) {
        uint32_t b = bitmask[(size_t)pix * Wk + w];
        t.sbits[(size_t)w * n_samples + s] = b;
        pc += __popc(b);
    }
    t.spop[s] = pc;
}

// one thread per (label, code index j)
__global__ void majority_kernel(const int32_t* __restrict__ off, int n_labels, int k, int Wk,
                                int n_samples, const uint32_t* __restrict__ sbits,
                                uint32_t* __restrict__ rep) {
    int tid = blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= n_labels * Wk * 32) return;
    const int i = tid / (Wk * 32), j = tid % (Wk * 32);
    const int w = j >> 5, b = j & 31;
    int cnt = 0;
    const int m = off[i + 1] - off[i];
    for (int s = off[i]; s < off[i + 1]; ++s) cnt += (sbits[(size_t)w * n_samples + s] >> b) & 1;
    const bool set = (j < k) && (2 * cnt >= m);
    const unsigned word = __ballot_sync(0xffffffffu, set);  // 32 consecutive j share a word
    if (b == 0) rep[(size_t)i * Wk + w] = word;
}

__global__ void set_offsets_kernel(OffsetsParam p, int n, int32_t* __restrict__ dst) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = p.v[i];
}

}  // namespace

cudaError_t launch_set_offsets(const OffsetsParam& p, int n, int32_t* dst, cudaStream_t st) {
    set_offsets_kernel<<<1, 128, 0, st>>>(p, n, dst);
    return cudaGetLastError();
}

cudaError_t launch_edt(const EdtArgs& a, cudaStream_t st) {
    const int Wb = (a.W + 31) / 32;
    const long long nrow = (long long)a.n_labels * a.H;
    cudaError_t e = cudaMemsetAsync(a.seedbits, 0, sizeof(uint32_t) * nrow * Wb, st);
    if (e != cudaSuccess) return e;
    seed_kernel<<<(a.n_samples + 255) / 256, 256, 0, st>>>(a.d_label_off, a.n_labels,
                                                           a.sample_pix, a.n_samples, a.H, a.W,
                                                           a.seedbits, a.d_err);
    rows_binary_kernel<<<(unsigned)((nrow * 32 + 127) / 128), 128, 0, st>>>(
        a.H, a.W, a.n_labels, a.seedbits, a.colbuf);
    const long long ncol = (long long)a.n_labels * a.W;
    if (ncol < 16384 && a.H <= 64) {
        // too few columns for the envelope pass to fill the GPU: scan per pixel
        const long long n = (long long)a.n_labels * a.H * a.W;
        cols_scan_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a.H, a.W, a.n_labels,
                                                                       a.colbuf, a.dist2);
        return cudaGetLastError();
    }
    // envelopes of 32 columns per block (S segments) in shared memory when they fit
    const unsigned nblk = (unsigned)((ncol + 31) / 32);
    auto run = [&](auto seg_c) -> cudaError_t {
        constexpr int S = decltype(seg_c)::value;
        const size_t smem = (size_t)((a.H + S - 1) / S) * S * 2 * sizeof(int32_t) * 32;
        if (smem <= 110u * 1024u) {
            cudaError_t e2 = cudaFuncSetAttribute(cols_envelope_split_kernel<true, S>,
                                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  (int)smem);
            if (e2 != cudaSuccess) return e2;
            cols_envelope_split_kernel<true, S><<<nblk, 32 * NSEG, smem, st>>>(
                a.H, a.W, a.n_labels, a.colbuf, nullptr, nullptr, a.dist2);
        } else {
            cols_envelope_split_kernel<false, S><<<nblk, 32 * NSEG, 0, st>>>(
                a.H, a.W, a.n_labels, a.colbuf, a.vbuf, a.fbuf, a.dist2);
        }
        return cudaSuccess;
    };
    // the fewest segments (2, 4 or 8) whose sweeps are at most 128 rows long
    e = a.H > 512 ? run(std::integral_constant<int, 8>{})
      : a.H > 256 ? run(std::integral_constant<int, 4>{})
                  : run(std::integral_constant<int, 2>{});
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_gather(const float* img, int H, int W, const uint32_t* bitmask, int k,
                          int n_labels, const int32_t* d_label_off, const int32_t* sample_pix,
                          int n_samples, bool want_rep, const SampleTables& t, cudaStream_t st) {
    const int Wk = (k + 31) / 32;
    gather_kernel<<<(n_samples + 255) / 256, 256, 0, st>>>(img, W, (long long)H * W, bitmask, Wk, sample_pix,
                                                           n_samples, t);
    if (want_rep) {
        int nthr = n_labels * Wk * 32;
        majority_kernel<<<(nthr + 127) / 128, 128, 0, st>>>(d_label_off, n_labels, k, Wk,
                                                            n_samples, t.sbits, t.rep);
    }
    return cudaGetLastError();
}
