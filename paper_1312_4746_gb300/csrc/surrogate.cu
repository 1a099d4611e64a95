// C ABI of the learned surrogate: fit (exact targets at a seeded pixel subset,
// standardisation, Adam training with the project's forward/backward
// kernels, calibration of the fallback gap on a held-out subset) and eval
// (network everywhere, exact sum on the low-margin pixels). Also the two
// kernel hooks cs_mlp_forward and cs_mlp_grad.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.h"

namespace {

// splitmix64 (Steele, Lea, Flood 2014): the counter-based generator behind the
// pixel subsets and their shuffle.
uint64_t splitmix64(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

constexpr int MAX_VAL = 20000;

struct Sel {
    std::vector<int32_t> train, val;
};

// Pixel q is a training pixel when u(q) < frac and a validation pixel when
// frac <= u(q) < frac + vfrac, u(q) = splitmix64(seed ^ q) / 2^64. The
// training list is then shuffled (Fisher-Yates driven by splitmix64).
Sel select_pixels(long long P, double frac, uint64_t seed) {
    Sel s;
    const double vfrac = std::min(0.01, (double)MAX_VAL / (double)P);
    for (long long q = 0; q < P; ++q) {
        const double u = (double)(splitmix64(seed ^ (uint64_t)q) >> 11) * 0x1.0p-53;
        if (u < frac)
            s.train.push_back((int32_t)q);
        else if (u < frac + vfrac)
            s.val.push_back((int32_t)q);
    }
    uint64_t st = seed ^ 0x5DEECE66Dull;
    for (size_t i = s.train.size(); i > 1; --i) {
        st = splitmix64(st);
        const size_t j = (size_t)(st % i);
        std::swap(s.train[i - 1], s.train[j]);
    }
    return s;
}

}  // namespace

// Inputs of the network for a feature set (0: [R, G, B, x/W, y/H, a_1..a_16];
// 1: those, log max(d_i, d_min) per label and 24 Fourier terms of x, y);
// 0 when the set cannot take n labels.
static int surrogate_nin(int feature_set, int n) {
    if (feature_set == CS_SURR_BASIC) return 21;
    if (feature_set == CS_SURR_EXTENDED) return 45 + n <= 64 ? 45 + n : 0;
    return 0;
}

// surrogate state kept in the context (allocated by the first fit)
static cs_status ensure_surrogate(cs_ctx* ctx, int nin, int n) {
    const int np = mlp_param_count(nin, n);
    // params | m | v | grads | stats (2 nin + 2 n) | eta | loss
    const size_t need = (size_t)4 * np + 2 * nin + 2 * n + 2;
    if (ctx->surr_buf && ctx->surr_cap >= need) return CS_OK;
    if (ctx->surr_buf) cudaFree(ctx->surr_buf);
    ctx->surr_buf = nullptr;
    ctx->surr_cap = 0;
    ctx->surr_ready = false;
    if (cudaMalloc(&ctx->surr_buf, need * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        return cs_set_error(ctx, CS_ERR_NOMEM, "surrogate state allocation failed");
    }
    ctx->surr_cap = need;
    return CS_OK;
}

// Network scratch in the context: the kernels' weight image, then the
// per-CTA gradient sums of one training step (G CTAs).
struct MlpScratch {
    unsigned char* image;
    float* part;
};
static cs_status mlp_scratch(cs_ctx* ctx, int nin, int n, int G, MlpScratch& out) {
    const size_t img = (mlp_image_bytes(nin, n) + 255) & ~(size_t)255;
    const size_t floats = img / sizeof(float) + (size_t)G * mlp_part_stride(nin, n);
    if (!ctx->mlp_part || ctx->mlp_part_cap < floats) {
        if (ctx->mlp_part) cudaFree(ctx->mlp_part);
        ctx->mlp_part = nullptr;
        ctx->mlp_part_cap = 0;
        if (cudaMalloc(&ctx->mlp_part, floats * sizeof(float)) != cudaSuccess) {
            cudaGetLastError();
            return cs_set_error(ctx, CS_ERR_NOMEM, "network scratch allocation failed");
        }
        ctx->mlp_part_cap = floats;
    }
    out.image = reinterpret_cast<unsigned char*>(ctx->mlp_part);
    out.part = ctx->mlp_part + img / sizeof(float);
    return CS_OK;
}

struct SurrPtrs {
    float *p, *m, *v, *g, *stats, *eta, *loss;
};
static SurrPtrs surr_ptrs(cs_ctx* ctx, int nin, int n) {
    const int np = mlp_param_count(nin, n);
    SurrPtrs s;
    s.p = ctx->surr_buf;
    s.m = s.p + np;
    s.v = s.m + np;
    s.g = s.v + np;
    s.stats = s.g + np;
    s.eta = s.stats + 2 * nin + 2 * n;
    s.loss = s.eta + 1;
    return s;
}

extern "C" {

cs_status cs_mlp_forward(cs_ctx* ctx, const float* params, int n_in, int n_out, const float* X,
                         int rows, float* Z, void* stream) {
    const char* fn = "cs_mlp_forward";
    if (!ctx) return cs_set_error(nullptr, CS_ERR_INVALID_ARG, "%s: ctx is NULL", fn);
    if (!params || !X || !Z || rows < 1 || n_in < 1 || n_in > 64 || n_out < 1 ||
        n_out > CS_MAX_LABELS)
        return cs_set_error(ctx, CS_ERR_INVALID_ARG, "%s: bad arguments", fn);
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    MlpScratch ms;
    cs_status s = mlp_scratch(ctx, n_in, n_out, 0, ms);
    if (s) return s;
    cudaError_t e = launch_mlp_pack(params, n_in, n_out, ms.image, st);
    if (e == cudaSuccess)
        e = launch_mlp_forward(ms.image, n_in, n_out, X, rows, Z, ctx->n_sm, ctx->d_err,
                               ctx->wait_ns, st);
    if (e != cudaSuccess) return cs_set_error(ctx, CS_ERR_CUDA, "%s: %s", fn, cudaGetErrorString(e));
    return cs_check_launch(ctx, fn);
}

cs_status cs_mlp_grad(cs_ctx* ctx, const float* params, int n_in, int n_out, const float* X,
                      const float* T, int rows, float* grads, float* loss, void* stream) {
    const char* fn = "cs_mlp_grad";
    if (!ctx) return cs_set_error(nullptr, CS_ERR_INVALID_ARG, "%s: ctx is NULL", fn);
    if (!params || !X || !T || !grads || !loss || rows < 1 || n_in < 1 || n_in > 64 ||
        n_out < 1 || n_out > CS_MAX_LABELS)
        return cs_set_error(ctx, CS_ERR_INVALID_ARG, "%s: bad arguments", fn);
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int G = mlp_train_ctas(rows, ctx->n_sm);
    MlpScratch ms;
    cs_status s = mlp_scratch(ctx, n_in, n_out, G, ms);
    if (s) return s;
    cudaError_t e = launch_mlp_pack(params, n_in, n_out, ms.image, st);
    if (e == cudaSuccess)
        e = launch_mlp_train(ms.image, n_in, n_out, X, T, rows, 0, rows, ms.part, G, ctx->d_err,
                             ctx->wait_ns, st);
    if (e == cudaSuccess)
        e = launch_reduce_adam(ms.part, G, n_in, n_out, nullptr, grads, nullptr, nullptr, 0.f, 1,
                               loss, nullptr, st);
    if (e != cudaSuccess) return cs_set_error(ctx, CS_ERR_CUDA, "%s: %s", fn, cudaGetErrorString(e));
    return cs_check_launch(ctx, fn);
}

int cs_mlp_param_count(int n_in, int n_out) {
    return (n_in < 1 || n_in > 64 || n_out < 1) ? 0 : mlp_param_count(n_in, n_out);
}

cs_status cs_surrogate_fit(cs_ctx* ctx, const float* img, int H, int W, const uint32_t* bitmask,
                           const float* lead16, int k, int n_labels, const int32_t* label_off,
                           const int32_t* sample_pix, const cs_params* prm, double frac,
                           int steps, int features, uint64_t seed, void* stream) {
    const char* fn = "cs_surrogate_fit";
    if (!ctx) return cs_set_error(nullptr, CS_ERR_INVALID_ARG, "%s: ctx is NULL", fn);
    if (!img || !bitmask || !lead16 || !sample_pix)
        return cs_set_error(ctx, CS_ERR_INVALID_ARG, "%s: null required pointer", fn);
    if (!(frac > 0.0 && frac <= 0.5) || steps < 1)
        return cs_set_error(ctx, CS_ERR_INVALID_ARG, "%s: need 0 < frac <= 0.5 and steps >= 1", fn);
    cs_status s = cs_check_likelihood_args(ctx, fn, H, W, k, n_labels, label_off, prm);
    if (s) return s;
    const int n = n_labels, nin = surrogate_nin(features, n);
    if (nin == 0)
        return cs_set_error(ctx, CS_ERR_INVALID_ARG,
                            "%s: feature set %d is unknown or cannot take %d labels", fn, features, n);
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const long long P = (long long)H * W;
    Sel sel = select_pixels(P, frac, seed);
    const int ntr = (int)sel.train.size(), nva = (int)sel.val.size();
    if (ntr < 128 || nva < 1)
        return cs_set_error(ctx, CS_ERR_INVALID_ARG, "%s: image too small for frac=%g", fn, frac);
    const int N = ntr + nva;
    if ((s = ensure_surrogate(ctx, nin, n))) return s;
    const int batch = 128 * std::max(1, std::min(ctx->n_sm, (ntr + 127) / 128));
    const int G = mlp_train_ctas(batch, ctx->n_sm);
    MlpScratch ms;
    if ((s = mlp_scratch(ctx, nin, n, G, ms))) return s;

    // scratch: likelihood plan (distances, sample tables), list, targets, features
    LikPlanRef plan;
    cs_params exact = *prm;
    exact.precision = CS_FP32;
    size_t off_extra = 0;
    if ((s = cs_plan_likelihood(ctx, plan, H, W, k, n_labels, label_off, &exact, nullptr,
                                (size_t)N * sizeof(int32_t) + 256 +        // list
                                    (size_t)n * N * sizeof(float) + 256 +  // T (label-major)
                                    (size_t)N * nin * sizeof(float) + 256 + // X
                                    (size_t)N * n * sizeof(float) + 256 +  // standardised T
                                    (size_t)N * n * sizeof(float) + 256 +  // calibration output
                                    16,
                                &off_extra)))
        return s;
    Carve c(ctx->scratch);
    c.off = off_extra;
    int32_t* d_list = c.take<int32_t>(N);
    float* T = c.take<float>((size_t)n * N);
    float* X = c.take<float>((size_t)N * nin);
    float* Ts = c.take<float>((size_t)N * n);
    float* Z = c.take<float>((size_t)N * n);
    int* d_count = c.take<int>(1);
    std::vector<int32_t> hl(sel.train);
    hl.insert(hl.end(), sel.val.begin(), sel.val.end());
    cudaError_t e = cudaMemcpyAsync(d_list, hl.data(), sizeof(int32_t) * N, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_count, &N, sizeof(int), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cs_enqueue_exact_list(ctx, plan, img, bitmask, sample_pix, &exact,
                                                    d_list, d_count, N, T, nullptr, nullptr, st);
    SurrPtrs sp = surr_ptrs(ctx, nin, n);
    if (e == cudaSuccess)
        e = launch_features(img, lead16, cs_plan_dist2(plan), H, W, n, features, (float)prm->d_min,
                            nin, d_list, N, X, st);
    if (e == cudaSuccess) e = launch_stats(X, nin, T, n, N, ntr, sp.stats, st);
    if (e == cudaSuccess) e = launch_standardize(X, nin, T, n, N, N, sp.stats, Ts, st);
    if (e == cudaSuccess) e = launch_init_params(sp.p, sp.m, sp.v, nin, n, seed, st);
    if (e == cudaSuccess) e = launch_mlp_pack(sp.p, nin, n, ms.image, st);
    {
        StageTimer tm(ctx, CS_STAGE_TRAIN, st);
        for (int t = 0; e == cudaSuccess && t < steps; ++t) {
            e = launch_mlp_train(ms.image, nin, n, X, Ts, ntr, (long long)t * batch, batch, ms.part,
                                 G, ctx->d_err, ctx->wait_ns, st);
            // learning rate 4e-3, cosine decay to 1e-4
            const float lr = 1e-4f + 0.5f * (4e-3f - 1e-4f) * (1.f + cosf(3.14159265f * t / steps));
            if (e == cudaSuccess)
                e = launch_reduce_adam(ms.part, G, nin, n, sp.p, nullptr, sp.m, sp.v, lr, t + 1,
                                       sp.loss, ms.image, st);
        }
    }
    // calibration on the validation rows: largest log-likelihood error
    if (e == cudaSuccess) e = cudaMemsetAsync(sp.eta, 0, sizeof(float), st);
    if (e == cudaSuccess)
        e = launch_mlp_forward(ms.image, nin, n, X + (size_t)ntr * nin, nva, Z, ctx->n_sm,
                               ctx->d_err, ctx->wait_ns, st);
    if (e == cudaSuccess) e = launch_calib(Z, Ts + (size_t)ntr * n, nin, n, nva, sp.stats, sp.eta, st);
    if (e != cudaSuccess) return cs_set_error(ctx, CS_ERR_CUDA, "%s: %s", fn, cudaGetErrorString(e));
    ctx->surr_n = n;
    ctx->surr_nin = nin;
    ctx->surr_set = features;
    ctx->surr_ready = true;
    ctx->surr_train = ntr;
    ctx->surr_val = nva;
    return cs_check_launch(ctx, fn);
}

cs_status cs_surrogate_eval(cs_ctx* ctx, const float* img, int H, int W, const uint32_t* bitmask,
                            const float* lead16, int k, int n_labels, const int32_t* label_off,
                            const int32_t* sample_pix, const cs_params* prm, int rule,
                            double margin, float* neglog, float* post, int32_t* n_fallback,
                            void* stream) {
    const char* fn = "cs_surrogate_eval";
    if (!ctx) return cs_set_error(nullptr, CS_ERR_INVALID_ARG, "%s: ctx is NULL", fn);
    if (!img || !bitmask || !lead16 || !sample_pix || !neglog)
        return cs_set_error(ctx, CS_ERR_INVALID_ARG, "%s: null required pointer", fn);
    if (!ctx->surr_ready || ctx->surr_n != n_labels)
        return cs_set_error(ctx, CS_ERR_INVALID_ARG, "%s: no surrogate fitted for %d labels", fn,
                            n_labels);
    if (!(margin >= 0.0 && margin <= 1.0))
        return cs_set_error(ctx, CS_ERR_INVALID_ARG, "%s: margin must lie in [0, 1]", fn);
    if (rule < CS_FALLBACK_GUARANTEED || rule > CS_FALLBACK_NONE)
        return cs_set_error(ctx, CS_ERR_INVALID_ARG, "%s: unknown fallback rule %d", fn, rule);
    cs_status s = cs_check_likelihood_args(ctx, fn, H, W, k, n_labels, label_off, prm);
    if (s) return s;
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const long long P = (long long)H * W;
    cs_params exact = *prm;
    exact.precision = CS_FP32;
    LikPlanRef plan;
    size_t off_extra = 0;
    if ((s = cs_plan_likelihood(ctx, plan, H, W, k, n_labels, label_off, &exact, nullptr,
                                (size_t)P * sizeof(int32_t) + 256 + 16, &off_extra)))
        return s;
    Carve c(ctx->scratch);
    c.off = off_extra;
    int32_t* fb_list = c.take<int32_t>(P);
    int* fb_count = c.take<int>(1);
    const int nin = ctx->surr_nin;
    SurrPtrs sp = surr_ptrs(ctx, nin, n_labels);
    MlpScratch ms;
    if ((s = mlp_scratch(ctx, nin, n_labels, 0, ms))) return s;
    cudaError_t e = cudaMemsetAsync(fb_count, 0, sizeof(int), st);
    if (e == cudaSuccess) e = launch_mlp_pack(sp.p, nin, n_labels, ms.image, st);
    if (e == cudaSuccess) e = cs_enqueue_prepare(ctx, plan, img, bitmask, sample_pix, &exact, st);
    if (e == cudaSuccess) {
        SurrogateEvalArgs a{};
        a.image = ms.image;
        a.nin = nin;
        a.n = n_labels;
        a.feature_set = ctx->surr_set;
        a.stats = sp.stats;
        a.eta = sp.eta;
        a.img = img;
        a.lead16 = lead16;
        a.H = H;
        a.W = W;
        a.dist2 = cs_plan_dist2(plan);
        a.label_off = cs_plan_label_off(plan);
        a.bitmask = bitmask;
        a.rep = cs_plan_rep(plan);
        a.Wk = (k + 31) / 32;
        a.mode = prm->mode;
        a.alpha = (float)prm->alpha;
        a.d_min = (float)prm->d_min;
        a.kappa_beta = (float)prm->kappa_beta;
        a.sigma_c2 = (float)prm->sigma_c2;
        a.rho_var = prm->rho_variance != 0;
        a.rule = rule;
        a.margin = (float)margin;
        a.eps = 0.005f;
        a.neglog = neglog;
        a.post = post;
        a.fb_list = fb_list;
        a.fb_count = fb_count;
        a.n_sm = ctx->n_sm;
        a.d_err = ctx->d_err;
        a.wait_ns = ctx->wait_ns;
        StageTimer tm(ctx, CS_STAGE_SURROGATE, st);
        e = launch_surrogate_eval(a, st);
    }
    if (e == cudaSuccess)
        e = cs_enqueue_exact_list_prepared(ctx, plan, img, bitmask, &exact, fb_list, fb_count,
                                           (int)P, nullptr, neglog, post, st);
    if (e == cudaSuccess && n_fallback) {
        e = cudaMemcpyAsync(n_fallback, fb_count, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    if (e != cudaSuccess) return cs_set_error(ctx, CS_ERR_CUDA, "%s: %s", fn, cudaGetErrorString(e));
    return cs_check_launch(ctx, fn);
}

cs_status cs_surrogate_params(cs_ctx* ctx, float* host_params, int cap, int* n_params) {
    if (!ctx || !n_params) return cs_set_error(ctx, CS_ERR_INVALID_ARG, "cs_surrogate_params: bad arguments");
    if (!ctx->surr_ready) return cs_set_error(ctx, CS_ERR_INVALID_ARG, "cs_surrogate_params: no surrogate");
    const int np = mlp_param_count(ctx->surr_nin, ctx->surr_n);
    *n_params = np;
    if (!host_params) return CS_OK;
    if (cap < np) return cs_set_error(ctx, CS_ERR_INVALID_ARG, "cs_surrogate_params: cap < %d", np);
    DeviceGuard g(ctx->device);
    if (cudaMemcpy(host_params, ctx->surr_buf, sizeof(float) * np, cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return cs_set_error(ctx, CS_ERR_CUDA, "cs_surrogate_params: copy failed");
    }
    return CS_OK;
}

// File: "CSSURR02", int32 n_labels, n_in, feature set, n_params, n_train,
// n_val, then float32 params[n_params], stats[2 n_in + 2 n], eta, loss
// (host byte order).
static const char SURR_MAGIC[8] = {'C', 'S', 'S', 'U', 'R', 'R', '0', '2'};

cs_status cs_surrogate_save(cs_ctx* ctx, const char* path) {
    const char* fn = "cs_surrogate_save";
    if (!ctx) return cs_set_error(nullptr, CS_ERR_INVALID_ARG, "%s: ctx is NULL", fn);
    if (!path) return cs_set_error(ctx, CS_ERR_INVALID_ARG, "%s: path is NULL", fn);
    if (!ctx->surr_ready) return cs_set_error(ctx, CS_ERR_INVALID_ARG, "%s: no surrogate", fn);
    DeviceGuard g(ctx->device);
    const int n = ctx->surr_n, nin = ctx->surr_nin, np = mlp_param_count(nin, n);
    const int ns = 2 * nin + 2 * n;
    std::vector<float> buf((size_t)np + ns + 2);
    SurrPtrs sp = surr_ptrs(ctx, nin, n);
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(buf.data(), sp.p, sizeof(float) * np, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess)
        e = cudaMemcpy(buf.data() + np, sp.stats, sizeof(float) * (ns + 2), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cs_set_error(ctx, CS_ERR_CUDA, "%s: %s", fn, cudaGetErrorString(e));
    }
    FILE* f = std::fopen(path, "wb");
    if (!f) return cs_set_error(ctx, CS_ERR_INVALID_ARG, "%s: cannot open %s", fn, path);
    const int32_t hdr[6] = {n, nin, ctx->surr_set, np, ctx->surr_train, ctx->surr_val};
    const bool ok = std::fwrite(SURR_MAGIC, 1, 8, f) == 8 && std::fwrite(hdr, sizeof hdr, 1, f) == 1 &&
                    std::fwrite(buf.data(), sizeof(float), buf.size(), f) == buf.size();
    const bool closed = std::fclose(f) == 0;
    if (!ok || !closed) return cs_set_error(ctx, CS_ERR_INVALID_ARG, "%s: write to %s failed", fn, path);
    return CS_OK;
}

cs_status cs_surrogate_load(cs_ctx* ctx, const char* path) {
    const char* fn = "cs_surrogate_load";
    if (!ctx) return cs_set_error(nullptr, CS_ERR_INVALID_ARG, "%s: ctx is NULL", fn);
    if (!path) return cs_set_error(ctx, CS_ERR_INVALID_ARG, "%s: path is NULL", fn);
    FILE* f = std::fopen(path, "rb");
    if (!f) return cs_set_error(ctx, CS_ERR_INVALID_ARG, "%s: cannot open %s", fn, path);
    char magic[8];
    int32_t hdr[6];
    bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, SURR_MAGIC, 8) == 0 &&
              std::fread(hdr, sizeof hdr, 1, f) == 1;
    const int n = ok ? hdr[0] : 0, nin = ok ? hdr[1] : 0;
    ok = ok && n >= 1 && n <= CS_MAX_LABELS && nin == surrogate_nin(hdr[2], n) && nin > 0 &&
         hdr[3] == mlp_param_count(nin, n) && hdr[4] >= 0 && hdr[5] >= 0;
    std::vector<float> buf;
    if (ok) {
        buf.resize((size_t)hdr[3] + 2 * nin + 2 * n + 2);
        ok = std::fread(buf.data(), sizeof(float), buf.size(), f) == buf.size();
    }
    std::fclose(f);
    if (!ok) return cs_set_error(ctx, CS_ERR_INVALID_ARG, "%s: %s is not a surrogate file", fn, path);
    DeviceGuard g(ctx->device);
    cs_status s = ensure_surrogate(ctx, nin, n);
    if (s) return s;
    const int np = hdr[3], ns = 2 * nin + 2 * n;
    SurrPtrs sp = surr_ptrs(ctx, nin, n);
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(sp.p, buf.data(), sizeof(float) * np, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(sp.stats, buf.data() + np, sizeof(float) * (ns + 2), cudaMemcpyHostToDevice);
    // fresh optimiser state: a later fit starts from these weights' values
    if (e == cudaSuccess) e = cudaMemset(sp.m, 0, sizeof(float) * 3 * (size_t)np);
    if (e != cudaSuccess) {
        cudaGetLastError();
        ctx->surr_ready = false;
        return cs_set_error(ctx, CS_ERR_CUDA, "%s: %s", fn, cudaGetErrorString(e));
    }
    ctx->surr_n = n;
    ctx->surr_nin = nin;
    ctx->surr_set = hdr[2];
    ctx->surr_train = hdr[4];
    ctx->surr_val = hdr[5];
    ctx->surr_ready = true;
    return CS_OK;
}

cs_status cs_surrogate_info(cs_ctx* ctx, float* host_stats, int cap, float* eta, float* loss,
                            int* n_train, int* n_val, int* n_in) {
    if (!ctx) return cs_set_error(nullptr, CS_ERR_INVALID_ARG, "cs_surrogate_info: ctx is NULL");
    if (!ctx->surr_ready) return cs_set_error(ctx, CS_ERR_INVALID_ARG, "cs_surrogate_info: no surrogate");
    DeviceGuard g(ctx->device);
    const int n = ctx->surr_n, nin = ctx->surr_nin;
    SurrPtrs sp = surr_ptrs(ctx, nin, n);
    if (host_stats) {
        if (cap < 2 * nin + 2 * n)
            return cs_set_error(ctx, CS_ERR_INVALID_ARG, "cs_surrogate_info: cap < %d", 2 * nin + 2 * n);
        if (cudaMemcpy(host_stats, sp.stats, sizeof(float) * (2 * nin + 2 * n), cudaMemcpyDeviceToHost) != cudaSuccess)
            return cs_set_error(ctx, CS_ERR_CUDA, "cs_surrogate_info: copy failed");
    }
    if (eta && cudaMemcpy(eta, sp.eta, sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
        return cs_set_error(ctx, CS_ERR_CUDA, "cs_surrogate_info: copy failed");
    if (loss && cudaMemcpy(loss, sp.loss, sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
        return cs_set_error(ctx, CS_ERR_CUDA, "cs_surrogate_info: copy failed");
    if (n_train) *n_train = ctx->surr_train;
    if (n_val) *n_val = ctx->surr_val;
    if (n_in) *n_in = nin;
    return CS_OK;
}

}  // extern "C"
