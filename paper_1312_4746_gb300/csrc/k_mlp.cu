// Learned surrogate of the data term: a 21 -> 64 -> 64 -> 64 -> n MLP (SiLU)
// that predicts, per pixel and label, the log kernel sum
//   T_i(x) = log sum_j k_rho(x - x_ij) k_sigma(I - I_ij) [exp(-TSM / beta)]
// of Sec. 3.1 (Eq. color, Eq. post_text); L_i then follows exactly from the
// scribble distance transform. Weights are used in bf16 (rounded from fp32
// masters); all arithmetic is fp32.
//
// Parameter vector (fp32), n = number of labels:
//   W1 [64][21] | b1 [64] | W2 [64][64] | b2 [64] | W3 [64][64] | b3 [64] | W4 [n][64] | b4 [n]
//
// mlp_train_kernel: one block of 64 threads = 64 samples of a minibatch; the
//   bf16-rounded weights and per-sample activations (h_l) and SiLU derivatives
//   (g_l) sit in shared memory; after the forward pass each thread forms its
//   output error, back-propagates it, and the block forms the weight
//   gradients as small GEMMs over its 64 samples, accumulated into a global
//   gradient vector with atomics (loss = mean (z - t)^2 / 2 over batch and labels).
// adam_kernel: bias-corrected Adam on the fp32 masters, clears the gradient.
// mlp_eval_kernel: forward pass per pixel from raw features, then
//   L_i = sd_t,i z_i + mu_t,i - log m_i - log(2 pi s2_i) - 1.5 log(2 pi sigma_c2)
//   (s2_i = rho_i^2, or rho_i when rho is read as the location variance)
//   (+ the factorised texture log-posterior), posteriors, and the fallback
//   decision (top-2 posterior margin below `margin`, or top-2 log-likelihood
//   gap below the calibrated `gap_min`): such pixels are appended to a list
//   that the exact sum then overwrites.
#include <cuda_bf16.h>

#include <cstdint>

#include "internal.h"

namespace {

constexpr int NIN = 21, HID = 64, BS = 64, SP = BS + 1;  // SP: padded sample stride

__host__ __device__ constexpr int off_W1() { return 0; }
__host__ __device__ constexpr int off_b1() { return HID * NIN; }
__host__ __device__ constexpr int off_W2() { return off_b1() + HID; }
__host__ __device__ constexpr int off_b2() { return off_W2() + HID * HID; }
__host__ __device__ constexpr int off_W3() { return off_b2() + HID; }
__host__ __device__ constexpr int off_b3() { return off_W3() + HID * HID; }
__host__ __device__ constexpr int off_W4() { return off_b3() + HID; }
__host__ __device__ inline int off_b4(int n) { return off_W4() + n * HID; }

__device__ __forceinline__ float bf16r(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }
__device__ __forceinline__ float sigm(float u) { return 1.f / (1.f + __expf(-u)); }

// weights (bf16-rounded) into shared memory
__device__ __forceinline__ void load_weights(const float* __restrict__ params, int np, float* sw) {
    for (int i = threadIdx.x; i < np; i += blockDim.x) sw[i] = bf16r(params[i]);
}

// z = W4 silu(W3 silu(W2 silu(W1 x + b1) + b2) + b3) + b4 for one sample in
// registers; optional per-sample shared buffers receive h_l and silu'(u_l).
template <bool STORE>
__device__ __forceinline__ void forward_one(const float* sw, const float (&x)[NIN], int n,
                                            float* H1, float* H2, float* H3, float* G1, float* G2,
                                            float* G3, int s, float* z) {
    float h[HID], a[HID];
    const float* W1 = sw + off_W1();
#pragma unroll
    for (int j = 0; j < HID; ++j) {
        float acc = sw[off_b1() + j];
#pragma unroll
        for (int kk = 0; kk < NIN; ++kk) acc = fmaf(W1[j * NIN + kk], x[kk], acc);
        const float sg = sigm(acc);
        h[j] = acc * sg;
        if (STORE) {
            H1[j * SP + s] = h[j];
            G1[j * SP + s] = sg * (1.f + acc * (1.f - sg));
        }
    }
    for (int layer = 0; layer < 2; ++layer) {
        const float* Wl = sw + (layer == 0 ? off_W2() : off_W3());
        const float* bl = sw + (layer == 0 ? off_b2() : off_b3());
#pragma unroll
        for (int j = 0; j < HID; ++j) a[j] = bl[j];
        for (int kk = 0; kk < HID; ++kk) {
            const float hk = h[kk];
#pragma unroll
            for (int j = 0; j < HID; ++j) a[j] = fmaf(Wl[j * HID + kk], hk, a[j]);
        }
        float* Hs = layer == 0 ? H2 : H3;
        float* Gs = layer == 0 ? G2 : G3;
#pragma unroll
        for (int j = 0; j < HID; ++j) {
            const float sg = sigm(a[j]);
            h[j] = a[j] * sg;
            if (STORE) {
                Hs[j * SP + s] = h[j];
                Gs[j * SP + s] = sg * (1.f + a[j] * (1.f - sg));
            }
        }
    }
    const float* W4 = sw + off_W4();
    for (int j = 0; j < n; ++j) {
        float acc = sw[off_b4(n) + j];
#pragma unroll
        for (int kk = 0; kk < HID; ++kk) acc = fmaf(W4[j * HID + kk], h[kk], acc);
        z[j] = acc;
    }
}

// Block-local weight gradient: grad[j][c] += sum_s D[j][s] * A[c][s] for
// j < rows, c < cols (thread c owns column c).
__device__ __forceinline__ void wgrad(const float* D, const float* A, int rows, int cols,
                                      float* __restrict__ gW, float* __restrict__ gb) {
    const int c = threadIdx.x;
    if (c < cols) {
        float av[BS];
#pragma unroll
        for (int s = 0; s < BS; ++s) av[s] = A[c * SP + s];
        for (int j = 0; j < rows; ++j) {
            float acc = 0.f;
#pragma unroll
            for (int s = 0; s < BS; ++s) acc = fmaf(D[j * SP + s], av[s], acc);
            atomicAdd(gW + j * cols + c, acc);
        }
    }
    for (int j = threadIdx.x; j < rows; j += blockDim.x) {
        float acc = 0.f;
        for (int s = 0; s < BS; ++s) acc += D[j * SP + s];
        atomicAdd(gb + j, acc);
    }
}

// X: rows of standardised features; T: standardised targets [row][n];
// rows taken as (start + b) mod n_rows for b < batch (batch a multiple of 64).
__global__ void __launch_bounds__(BS) mlp_train_kernel(const float* __restrict__ params, int n,
                                                     const float* __restrict__ X,
                                                     const float* __restrict__ T, int n_rows,
                                                     long long start, int batch,
                                                     float* __restrict__ grads,
                                                     float* __restrict__ loss_acc) {
    extern __shared__ float smem[];
    const int np = off_b4(n) + n;
    float* sw = smem;
    float* H1 = sw + ((np + 3) & ~3);
    float* H2 = H1 + HID * SP;
    float* H3 = H2 + HID * SP;
    float* G1 = H3 + HID * SP;
    float* G2 = G1 + HID * SP;
    float* G3 = G2 + HID * SP;
    float* DZ = G3 + HID * SP;   // [n][SP]
    float* XS = DZ + 64 * SP;    // [21][SP]
    load_weights(params, np, sw);
    __syncthreads();
    const int s = threadIdx.x;
    const long long row = (start + (long long)blockIdx.x * BS + s) % n_rows;
    float x[NIN];
#pragma unroll
    for (int kk = 0; kk < NIN; ++kk) {
        x[kk] = X[row * NIN + kk];
        XS[kk * SP + s] = x[kk];
    }
    float z[64];
    forward_one<true>(sw, x, n, H1, H2, H3, G1, G2, G3, s, z);
    const float inv = 1.f / ((float)batch * (float)n);
    float l = 0.f;
    for (int j = 0; j < n; ++j) {
        const float d = z[j] - T[row * n + j];
        l += d * d;
        DZ[j * SP + s] = d * inv;
    }
    atomicAdd(loss_acc, 0.5f * l * inv);
    __syncthreads();
    // output layer gradients
    wgrad(DZ, H3, n, HID, grads + off_W4(), grads + off_b4(n));
    // delta of layer 3 (in place over G3): g3 * W4^T dz
    {
        const float* W4 = sw + off_W4();
        for (int kk = 0; kk < HID; ++kk) {
            float acc = 0.f;
            for (int j = 0; j < n; ++j) acc = fmaf(DZ[j * SP + s], W4[j * HID + kk], acc);
            G3[kk * SP + s] *= acc;
        }
    }
    __syncthreads();
    wgrad(G3, H2, HID, HID, grads + off_W3(), grads + off_b3());
    {
        const float* W3 = sw + off_W3();
        for (int kk = 0; kk < HID; ++kk) {
            float acc = 0.f;
            for (int j = 0; j < HID; ++j) acc = fmaf(G3[j * SP + s], W3[j * HID + kk], acc);
            G2[kk * SP + s] *= acc;
        }
    }
    __syncthreads();
    wgrad(G2, H1, HID, HID, grads + off_W2(), grads + off_b2());
    {
        const float* W2 = sw + off_W2();
        for (int kk = 0; kk < HID; ++kk) {
            float acc = 0.f;
            for (int j = 0; j < HID; ++j) acc = fmaf(G2[j * SP + s], W2[j * HID + kk], acc);
            G1[kk * SP + s] *= acc;
        }
    }
    __syncthreads();
    wgrad(G1, XS, HID, NIN, grads + off_W1(), grads + off_b1());
}

__global__ void adam_kernel(float* __restrict__ p, float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int np, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    g[i] = 0.f;
}

// forward pass only, for rows of standardised features (test hook and calibration)
__global__ void __launch_bounds__(BS) mlp_forward_kernel(const float* __restrict__ params, int n,
                                                       const float* __restrict__ X, int rows,
                                                       float* __restrict__ Z) {
    extern __shared__ float smem[];
    const int np = off_b4(n) + n;
    load_weights(params, np, smem);
    __syncthreads();
    const long long r = (long long)blockIdx.x * BS + threadIdx.x;
    if (r >= rows) return;
    float x[NIN];
#pragma unroll
    for (int kk = 0; kk < NIN; ++kk) x[kk] = X[r * NIN + kk];
    float z[64];
    forward_one<false>(smem, x, n, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, 0, z);
    for (int j = 0; j < n; ++j) Z[r * n + j] = z[j];
}

}  // namespace

int mlp_param_count(int n) { return off_b4(n) + n; }

size_t mlp_train_smem(int n) {
    const int np = off_b4(n) + n;
    return sizeof(float) * ((size_t)((np + 3) & ~3) + 6 * HID * SP + 64 * SP + NIN * SP);
}

cudaError_t launch_mlp_train(const float* params, int n, const float* X, const float* T,
                             int n_rows, long long start, int batch, float* grads,
                             float* loss_acc, cudaStream_t st) {
    const size_t smem = mlp_train_smem(n);
    cudaError_t e = cudaFuncSetAttribute(mlp_train_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    mlp_train_kernel<<<batch / BS, BS, smem, st>>>(params, n, X, T, n_rows, start, batch, grads,
                                                   loss_acc);
    return cudaGetLastError();
}

cudaError_t launch_adam(float* p, float* g, float* m, float* v, int np, float lr, int t,
                        cudaStream_t st) {
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
    adam_kernel<<<(np + 255) / 256, 256, 0, st>>>(p, g, m, v, np, lr, b1, b2, 1e-8f, c1, c2);
    return cudaGetLastError();
}

cudaError_t launch_mlp_forward(const float* params, int n, const float* X, int rows, float* Z,
                               cudaStream_t st) {
    const size_t smem = sizeof(float) * (size_t)mlp_param_count(n);
    cudaError_t e = cudaFuncSetAttribute(mlp_forward_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    mlp_forward_kernel<<<(rows + BS - 1) / BS, BS, smem, st>>>(params, n, X, rows, Z);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ data preparation

namespace {

// raw features of listed pixels: [R, G, B, x / W, y / H, a_1 .. a_16]
__global__ void features_kernel(const float* __restrict__ img, const float* __restrict__ lead16,
                                int H, int W, const int32_t* __restrict__ list, int rows,
                                float* __restrict__ X) {
    const long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (r >= rows) return;
    const long long q = list[r];
    float* x = X + r * NIN;
    x[0] = img[q * 3 + 0];
    x[1] = img[q * 3 + 1];
    x[2] = img[q * 3 + 2];
    x[3] = (float)(q % W) / (float)W;
    x[4] = (float)(q / W) / (float)H;
#pragma unroll
    for (int j = 0; j < 16; ++j) x[5 + j] = lead16[q * 16 + j];
}

// one block per column: mean and standard deviation over the first n_rows
// rows, in double, deterministic tree reduction. Columns 0..20 come from X
// (row-major, stride 21); columns 21..21+n-1 from T (label-major, stride cap).
__global__ void stats_kernel(const float* __restrict__ X, const float* __restrict__ T, int n,
                             int cap, int n_rows, float* __restrict__ stats) {
    __shared__ double red[2][256];
    const int c = blockIdx.x;
    double s = 0.0, s2 = 0.0;
    for (int r = threadIdx.x; r < n_rows; r += blockDim.x) {
        const double v = c < NIN ? (double)X[(size_t)r * NIN + c] : (double)T[(size_t)(c - NIN) * cap + r];
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
        // layout: mu_x[21] sd_x[21] mu_t[n] sd_t[n]
        if (c < NIN) {
            stats[c] = (float)mu;
            stats[NIN + c] = (float)sd;
        } else {
            stats[2 * NIN + (c - NIN)] = (float)mu;
            stats[2 * NIN + n + (c - NIN)] = (float)sd;
        }
    }
}

// X <- (X - mu_x) / sd_x in place; Ts[r][j] = (T[j][r] - mu_t,j) / sd_t,j
__global__ void standardize_kernel(float* __restrict__ X, const float* __restrict__ T, int n,
                                   int cap, int rows, const float* __restrict__ stats,
                                   float* __restrict__ Ts) {
    const long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (r >= rows) return;
    for (int c = 0; c < NIN; ++c) X[r * NIN + c] = (X[r * NIN + c] - stats[c]) / stats[NIN + c];
    for (int j = 0; j < n; ++j)
        Ts[r * n + j] = (T[(size_t)j * cap + r] - stats[2 * NIN + j]) / stats[2 * NIN + n + j];
}

__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

// Glorot-uniform weights from a counter-based generator, zero biases, zero
// optimiser state and gradients.
__global__ void init_params_kernel(float* __restrict__ p, float* __restrict__ m,
                                   float* __restrict__ v, float* __restrict__ g, int n,
                                   uint64_t seed) {
    const int np = off_b4(n) + n;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    float w = 0.f;
    int fan_in = 0, fan_out = 0;
    if (i < off_b1()) { fan_in = NIN; fan_out = HID; }
    else if (i >= off_W2() && i < off_b2()) { fan_in = HID; fan_out = HID; }
    else if (i >= off_W3() && i < off_b3()) { fan_in = HID; fan_out = HID; }
    else if (i >= off_W4() && i < off_b4(n)) { fan_in = HID; fan_out = n; }
    if (fan_in) {
        const double u = (double)(splitmix64(seed ^ (0xA5A5A5A5ull + (uint64_t)i)) >> 11) * 0x1.0p-53;
        const double lim = sqrt(6.0 / (fan_in + fan_out));
        w = (float)((2.0 * u - 1.0) * lim);
    }
    p[i] = w;
    m[i] = 0.f;
    v[i] = 0.f;
    g[i] = 0.f;
}

// largest |z - t| * sd_t over rows and labels (a positive float: max via int bits)
__global__ void calib_kernel(const float* __restrict__ Z, const float* __restrict__ Ts, int n,
                             int rows, const float* __restrict__ stats, float* __restrict__ eta) {
    const long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (r >= rows) return;
    float mx = 0.f;
    for (int j = 0; j < n; ++j)
        mx = fmaxf(mx, fabsf(Z[r * n + j] - Ts[r * n + j]) * stats[2 * NIN + n + j]);
    atomicMax(reinterpret_cast<int*>(eta), __float_as_int(mx));
}

// surrogate evaluation over all pixels (see the file header)
__global__ void __launch_bounds__(BS) surrogate_eval_kernel(
    const float* __restrict__ params, int n, const float* __restrict__ stats,
    const float* __restrict__ eta, const float* __restrict__ img, const float* __restrict__ lead16,
    int H, int W, const int32_t* __restrict__ dist2, const int32_t* __restrict__ label_off,
    const uint32_t* __restrict__ bitmask, const uint32_t* __restrict__ rep, int Wk, int mode,
    float alpha, float d_min, float kappa_beta, float sigma_c2, bool rho_var, float margin,
    float eps, float* __restrict__ neglog, float* __restrict__ post, int32_t* __restrict__ fb_list,
    int* __restrict__ fb_count) {
    extern __shared__ float smem[];
    const int np = off_b4(n) + n;
    load_weights(params, np, smem);
    __syncthreads();
    const long long P = (long long)H * W;
    const long long q = (long long)blockIdx.x * BS + threadIdx.x;
    if (q >= P) return;
    float x[NIN];
    x[0] = img[q * 3 + 0];
    x[1] = img[q * 3 + 1];
    x[2] = img[q * 3 + 2];
    x[3] = (float)(q % W) / (float)W;
    x[4] = (float)(q / W) / (float)H;
#pragma unroll
    for (int j = 0; j < 16; ++j) x[5 + j] = lead16[q * 16 + j];
#pragma unroll
    for (int c = 0; c < NIN; ++c) x[c] = (x[c] - stats[c]) / stats[NIN + c];
    float z[64];
    forward_one<false>(smem, x, n, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, 0, z);
    const float log_col_norm = 1.5f * logf(6.283185307179586f * sigma_c2);
    uint32_t bx[8];
    for (int w = 0; w < 8; ++w) bx[w] = (mode == CS_MODE_FACTORISED && w < Wk) ? bitmask[q * Wk + w] : 0u;
    // log-likelihoods, and the factorised texture posterior
    float tmax = -INFINITY;
    for (int j = 0; j < n; ++j) {
        const float rho = alpha * fmaxf(sqrtf((float)dist2[(size_t)j * P + q]), d_min);
        const float T = z[j] * stats[2 * NIN + n + j] + stats[2 * NIN + j];
        z[j] = T - logf((float)(label_off[j + 1] - label_off[j])) -
               logf(6.283185307179586f * (rho_var ? rho : rho * rho)) - log_col_norm;
        if (mode == CS_MODE_FACTORISED) {
            int h = 0;
            for (int w = 0; w < Wk; ++w) h += __popc(bx[w & 7] ^ rep[j * Wk + w]);
            tmax = fmaxf(tmax, -(float)h / (kappa_beta * rho));
        }
    }
    if (mode == CS_MODE_FACTORISED) {
        float ts = 0.f;
        for (int j = 0; j < n; ++j) {
            const float rho = alpha * fmaxf(sqrtf((float)dist2[(size_t)j * P + q]), d_min);
            int h = 0;
            for (int w = 0; w < Wk; ++w) h += __popc(bx[w & 7] ^ rep[j * Wk + w]);
            ts += expf(-(float)h / (kappa_beta * rho) - tmax);
        }
        const float tl = tmax + logf(ts);
        for (int j = 0; j < n; ++j) {
            const float rho = alpha * fmaxf(sqrtf((float)dist2[(size_t)j * P + q]), d_min);
            int h = 0;
            for (int w = 0; w < Wk; ++w) h += __popc(bx[w & 7] ^ rep[j * Wk + w]);
            z[j] += -(float)h / (kappa_beta * rho) - tl;
        }
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
    // a gap g guarantees a max probability error <= eps when every logit is
    // within eta of the truth: (n - 1) exp(-(g - 2 eta)) <= eps
    const float gap_min = 2.2f * (*eta) + logf(fmaxf((float)(n - 1), 1.f) / eps);
    // margin < 0: the network answers every pixel (no exact fallback)
    const bool fb = margin >= 0.f && ((p1 - p2 < margin) || (n > 1 && m1 - m2 < gap_min));
    if (fb) {
        const int idx = atomicAdd(fb_count, 1);
        if (idx < P) fb_list[idx] = (int32_t)q;
        return;
    }
    for (int j = 0; j < n; ++j) {
        neglog[(size_t)j * P + q] = -z[j];
        if (post) post[(size_t)j * P + q] = expf(z[j] - lse);
    }
}

}  // namespace

cudaError_t launch_features(const float* img, const float* lead16, int H, int W,
                            const int32_t* list, int rows, float* X, cudaStream_t st) {
    features_kernel<<<(rows + 127) / 128, 128, 0, st>>>(img, lead16, H, W, list, rows, X);
    return cudaGetLastError();
}

cudaError_t launch_stats(const float* X, const float* T, int n, int cap, int n_rows,
                         float* stats, cudaStream_t st) {
    stats_kernel<<<NIN + n, 256, 0, st>>>(X, T, n, cap, n_rows, stats);
    return cudaGetLastError();
}

cudaError_t launch_standardize(float* X, const float* T, int n, int cap, int rows,
                               const float* stats, float* Ts, cudaStream_t st) {
    standardize_kernel<<<(rows + 127) / 128, 128, 0, st>>>(X, T, n, cap, rows, stats, Ts);
    return cudaGetLastError();
}

cudaError_t launch_init_params(float* p, float* m, float* v, float* g, int n, uint64_t seed,
                               cudaStream_t st) {
    const int np = mlp_param_count(n);
    init_params_kernel<<<(np + 255) / 256, 256, 0, st>>>(p, m, v, g, n, seed);
    return cudaGetLastError();
}

cudaError_t launch_calib(const float* Z, const float* Ts, int n, int rows, const float* stats,
                         float* eta, cudaStream_t st) {
    calib_kernel<<<(rows + 127) / 128, 128, 0, st>>>(Z, Ts, n, rows, stats, eta);
    return cudaGetLastError();
}

cudaError_t launch_surrogate_eval(const SurrogateEvalArgs& a, cudaStream_t st) {
    const size_t smem = sizeof(float) * (size_t)mlp_param_count(a.n);
    cudaError_t e = cudaFuncSetAttribute(surrogate_eval_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const long long P = (long long)a.H * a.W;
    surrogate_eval_kernel<<<(unsigned)((P + BS - 1) / BS), BS, smem, st>>>(
        a.params, a.n, a.stats, a.eta, a.img, a.lead16, a.H, a.W, a.dist2, a.label_off,
        a.bitmask, a.rep, a.Wk, a.mode, a.alpha, a.d_min, a.kappa_beta, a.sigma_c2, a.rho_var,
        a.margin, a.eps, a.neglog, a.post, a.fb_list, a.fb_count);
    return cudaGetLastError();
}
