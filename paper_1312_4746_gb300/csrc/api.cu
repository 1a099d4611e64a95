// C ABI entry points: context, argument validation, scratch layout, launches.
#include <cstdarg>
#include <cstring>
#include <vector>

#include "internal.h"

#define CS_VERSION "cosparse-gb300 0.1 (sm_103a)"

static thread_local std::string g_noctx_err;

cs_status cs_set_error(cs_ctx* ctx, cs_status code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (ctx)
        ctx->err = buf;
    else
        g_noctx_err = buf;
    return code;
}

cs_status cs_check_launch(cs_ctx* ctx, const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return cs_set_error(ctx, CS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
    return CS_OK;
}

cs_status cs_ensure_scratch(cs_ctx* ctx, size_t bytes) {
    if (bytes <= ctx->scratch_cap) return CS_OK;
    size_t want = bytes + bytes / 4 + (1u << 20);
    if (ctx->scratch) {
        cudaFree(ctx->scratch);  // waits for outstanding work on the device
        ctx->scratch = nullptr;
        ctx->scratch_cap = 0;
    }
    cudaError_t e = cudaMalloc(&ctx->scratch, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cs_set_error(ctx, CS_ERR_NOMEM, "scratch allocation of %zu bytes failed: %s", want,
                            cudaGetErrorString(e));
    }
    ctx->scratch_cap = want;
    return CS_OK;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

static cudaEvent_t pool_get(cs_ctx* ctx) {
    if (!ctx->event_pool.empty()) {
        cudaEvent_t e = ctx->event_pool.back();
        ctx->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

StageTimer::StageTimer(cs_ctx* c, int s, cudaStream_t stream) : ctx(c), stage(s), st(stream) {
    if (!ctx->profiling) return;
    beg = pool_get(ctx);
    end = pool_get(ctx);
    if (beg) cudaEventRecord(beg, st);
}

StageTimer::~StageTimer() {
    if (!beg || !end) return;
    cudaEventRecord(end, st);
    ctx->records.push_back({stage, beg, end});
}

extern "C" {

const char* cs_version(void) { return CS_VERSION; }

cs_status cs_profile_enable(cs_ctx* ctx, int on) {
    if (!ctx) return cs_set_error(nullptr, CS_ERR_INVALID_ARG, "cs_profile_enable: ctx is NULL");
    ctx->profiling = on != 0;
    return CS_OK;
}

cs_status cs_profile_read(cs_ctx* ctx, int stage, double* ms, int* launches) {
    if (!ctx || !ms || !launches || stage < 0 || stage >= CS_N_STAGES)
        return cs_set_error(ctx, CS_ERR_INVALID_ARG, "cs_profile_read: bad arguments");
    DeviceGuard g(ctx->device);
    double tot = 0.0;
    int n = 0;
    std::vector<StageRecord> keep;
    for (const StageRecord& r : ctx->records) {
        if (r.stage != stage) {
            keep.push_back(r);
            continue;
        }
        float t = 0.f;
        if (cudaEventSynchronize(r.end) != cudaSuccess ||
            cudaEventElapsedTime(&t, r.beg, r.end) != cudaSuccess) {
            cudaError_t e = cudaGetLastError();
            return cs_set_error(ctx, CS_ERR_CUDA, "cs_profile_read: %s", cudaGetErrorString(e));
        }
        tot += t;
        ++n;
        ctx->event_pool.push_back(r.beg);
        ctx->event_pool.push_back(r.end);
    }
    ctx->records.swap(keep);
    *ms = tot;
    *launches = n;
    return CS_OK;
}

void cs_params_default(cs_params* out) {
    if (!out) return;
    memset(out, 0, sizeof *out);
    out->p = 7;
    out->mode = CS_MODE_PERSAMPLE;
    out->precision = CS_FP32;
    out->tau = 0.1;
    out->sigma_c2 = 1.3;
    out->alpha = 1.3;
    out->d_min = 1.0;
    out->kappa_beta = 1.0;
}

cs_status cs_create(cs_ctx** out, int device) {
    if (!out) return cs_set_error(nullptr, CS_ERR_INVALID_ARG, "cs_create: out is NULL");
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        return cs_set_error(nullptr, CS_ERR_INVALID_ARG, "cs_create: no CUDA device %d", device);
    }
    cs_ctx* c = new cs_ctx();
    c->device = device;
    DeviceGuard g(device);
    cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, device);
    if (cudaMalloc(&c->d_err, 2 * sizeof(int)) != cudaSuccess ||
        cudaMemset(c->d_err, 0, 2 * sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return cs_set_error(nullptr, CS_ERR_CUDA, "cs_create: cannot allocate the error word");
    }
    *out = c;
    return CS_OK;
}

void cs_destroy(cs_ctx* ctx) {
    if (!ctx) return;
    DeviceGuard g(ctx->device);
    cudaDeviceSynchronize();
    if (ctx->scratch) cudaFree(ctx->scratch);
    if (ctx->d_err) cudaFree(ctx->d_err);
    for (auto& r : ctx->records) {
        cudaEventDestroy(r.beg);
        cudaEventDestroy(r.end);
    }
    for (auto e : ctx->event_pool) cudaEventDestroy(e);
    delete ctx;
}

const char* cs_last_error(const cs_ctx* ctx) {
    return ctx ? ctx->err.c_str() : g_noctx_err.c_str();
}

cs_status cs_sync_status(cs_ctx* ctx, void* stream) {
    if (!ctx) return cs_set_error(nullptr, CS_ERR_INVALID_ARG, "cs_sync_status: ctx is NULL");
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess)
        return cs_set_error(ctx, CS_ERR_CUDA, "stream error: %s", cudaGetErrorString(e));
    int h[2] = {0, 0};
    e = cudaMemcpy(h, ctx->d_err, sizeof h, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess)
        return cs_set_error(ctx, CS_ERR_CUDA, "reading the error word: %s", cudaGetErrorString(e));
    if (h[0] == 0) return CS_OK;
    cudaMemset(ctx->d_err, 0, 2 * sizeof(int));
    if (h[0] == CS_DEVERR_TIMEOUT)
        return cs_set_error(ctx, CS_ERR_TIMEOUT, "a bounded device wait gave up (site %d)", h[1]);
    if (h[0] == CS_DEVERR_BAD_SAMPLE)
        return cs_set_error(ctx, CS_ERR_INVALID_ARG,
                            "sample %d has a pixel index outside the image (ignored)", h[1]);
    if (h[0] == CS_DEVERR_GUARD_FULL)
        return cs_set_error(ctx, CS_ERR_DEVICE,
                            "co-support guard list overflowed (%d entries needed); "
                            "bitmasks may be inexact",
                            h[1]);
    return cs_set_error(ctx, CS_ERR_DEVICE, "device error %d (detail %d)", h[0], h[1]);
}

// ---------------------------------------------------------------- cs_codes

static int guard_capacity(long long P, int k) {
    long long cap = P * (long long)k / 128 + 65536;
    if (cap > (1ll << 30)) cap = 1ll << 30;
    return (int)cap;
}

cs_status cs_codes(cs_ctx* ctx, const float* img, int H, int W, const float* omega, int k,
                   const float* mask, const cs_params* prm, float* codes, float* lead16,
                   uint32_t* bitmask, void* stream) {
    if (!ctx) return cs_set_error(nullptr, CS_ERR_INVALID_ARG, "cs_codes: ctx is NULL");
    if (!img || !omega || !mask || !prm)
        return cs_set_error(ctx, CS_ERR_INVALID_ARG, "cs_codes: null input pointer");
    if (H < 1 || W < 1 || H > CS_MAX_SIDE || W > CS_MAX_SIDE)
        return cs_set_error(ctx, CS_ERR_INVALID_ARG, "cs_codes: bad image size %dx%d", W, H);
    if (k < 1 || k > CS_MAX_K)
        return cs_set_error(ctx, CS_ERR_INVALID_ARG, "cs_codes: k=%d outside 1..%d", k, CS_MAX_K);
    if (!codes && !lead16 && !bitmask)
        return cs_set_error(ctx, CS_ERR_INVALID_ARG, "cs_codes: no output requested");
    if (prm->p < 1 || (prm->p & 1) == 0)
        return cs_set_error(ctx, CS_ERR_INVALID_ARG, "cs_codes: patch side %d is not odd", prm->p);
    if (prm->p < 3 || prm->p > 9)
        return cs_set_error(ctx, CS_ERR_UNSUPPORTED, "cs_codes: patch side %d not in 3..9",
                            prm->p);
    if (!(prm->tau >= 0.0))
        return cs_set_error(ctx, CS_ERR_INVALID_ARG, "cs_codes: tau must be >= 0");
    DeviceGuard g(ctx->device);
    long long P = (long long)H * W;
    int cap = guard_capacity(P, k);
    Carve m(nullptr);
    m.take<float>(k);
    m.take<int>(1);
    m.take<int2>(cap);
    if (!bitmask) m.take<uint32_t>(P * ((k + 31) / 32));
    cs_status s = cs_ensure_scratch(ctx, m.off);
    if (s) return s;
    Carve c(ctx->scratch);
    CodesArgs a{};
    a.img = img;
    a.H = H;
    a.W = W;
    a.omega = omega;
    a.k = k;
    a.mask = mask;
    a.p = prm->p;
    a.tau = prm->tau;
    a.codes = codes;
    a.lead16 = lead16;
    a.rownorm = c.take<float>(k);
    a.guard_count = c.take<int>(1);
    a.guard = c.take<int2>(cap);
    a.guard_cap = cap;
    a.bitmask = bitmask ? bitmask : c.take<uint32_t>(P * ((k + 31) / 32));
    a.d_err = ctx->d_err;
    cudaError_t e;
    {
        StageTimer tm(ctx, CS_STAGE_CODES, (cudaStream_t)stream);
        e = launch_codes_f32(a, (cudaStream_t)stream);
    }
    if (e != cudaSuccess) return cs_set_error(ctx, CS_ERR_CUDA, "cs_codes: %s", cudaGetErrorString(e));
    return cs_check_launch(ctx, "cs_codes");
}

cs_status cs_cosupport(cs_ctx* ctx, const float* codes, int P, int k, double tau,
                       uint32_t* bitmask, void* stream) {
    if (!ctx) return cs_set_error(nullptr, CS_ERR_INVALID_ARG, "cs_cosupport: ctx is NULL");
    if (!codes || !bitmask)
        return cs_set_error(ctx, CS_ERR_INVALID_ARG, "cs_cosupport: null pointer");
    if (P < 1 || k < 1 || k > CS_MAX_K)
        return cs_set_error(ctx, CS_ERR_INVALID_ARG, "cs_cosupport: bad shape P=%d k=%d", P, k);
    if (!(tau >= 0.0))
        return cs_set_error(ctx, CS_ERR_INVALID_ARG, "cs_cosupport: tau must be >= 0");
    DeviceGuard g(ctx->device);
    cudaError_t e = launch_cosupport(codes, P, k, tau, bitmask, (cudaStream_t)stream);
    if (e != cudaSuccess)
        return cs_set_error(ctx, CS_ERR_CUDA, "cs_cosupport: %s", cudaGetErrorString(e));
    return cs_check_launch(ctx, "cs_cosupport");
}

// ---------------------------------------------------------------- cs_likelihood

static cs_status check_labels(cs_ctx* ctx, const char* fn, int n_labels,
                              const int32_t* label_off) {
    if (n_labels < 1 || n_labels > CS_MAX_LABELS)
        return cs_set_error(ctx, CS_ERR_INVALID_ARG, "%s: n_labels=%d outside 1..%d", fn,
                            n_labels, CS_MAX_LABELS);
    if (!label_off) return cs_set_error(ctx, CS_ERR_INVALID_ARG, "%s: label_off is NULL", fn);
    if (label_off[0] != 0)
        return cs_set_error(ctx, CS_ERR_INVALID_ARG, "%s: label_off[0] must be 0", fn);
    for (int i = 0; i < n_labels; ++i)
        if (label_off[i + 1] - label_off[i] < 1)
            return cs_set_error(ctx, CS_ERR_INVALID_ARG, "%s: label %d has no scribble samples",
                                fn, i);
    return CS_OK;
}

static cs_status check_params(cs_ctx* ctx, const char* fn, const cs_params* prm) {
    if (!prm) return cs_set_error(ctx, CS_ERR_INVALID_ARG, "%s: params is NULL", fn);
    if (!(prm->sigma_c2 > 0) || !(prm->alpha > 0) || !(prm->d_min > 0) || !(prm->kappa_beta > 0))
        return cs_set_error(ctx, CS_ERR_INVALID_ARG,
                            "%s: sigma_c2, alpha, d_min and kappa_beta must be > 0", fn);
    if (prm->mode != CS_MODE_PERSAMPLE && prm->mode != CS_MODE_FACTORISED)
        return cs_set_error(ctx, CS_ERR_INVALID_ARG, "%s: unknown mode %d", fn, prm->mode);
    if (prm->precision != CS_FP32 && prm->precision != CS_BF16 && prm->precision != CS_FP8)
        return cs_set_error(ctx, CS_ERR_INVALID_ARG, "%s: unknown precision %d", fn,
                            prm->precision);
    return CS_OK;
}

cs_status cs_likelihood(cs_ctx* ctx, const float* img, int H, int W, const uint32_t* bitmask,
                        int k, int n_labels, const int32_t* label_off,
                        const int32_t* sample_pix, const cs_params* prm, int32_t* dist2,
                        float* neglog, float* post, void* stream) {
    const char* fn = "cs_likelihood";
    if (!ctx) return cs_set_error(nullptr, CS_ERR_INVALID_ARG, "%s: ctx is NULL", fn);
    if (!img || !bitmask || !sample_pix || !neglog)
        return cs_set_error(ctx, CS_ERR_INVALID_ARG, "%s: null required pointer", fn);
    if (H < 1 || W < 1 || H > CS_MAX_SIDE || W > CS_MAX_SIDE)
        return cs_set_error(ctx, CS_ERR_INVALID_ARG, "%s: bad image size %dx%d", fn, W, H);
    if (k < 1 || k > CS_MAX_K)
        return cs_set_error(ctx, CS_ERR_INVALID_ARG, "%s: k=%d outside 1..%d", fn, k, CS_MAX_K);
    cs_status s = check_labels(ctx, fn, n_labels, label_off);
    if (s) return s;
    s = check_params(ctx, fn, prm);
    if (s) return s;
    if (k > 256)
        return cs_set_error(ctx, CS_ERR_UNSUPPORTED, "%s: k=%d > 256 not supported yet", fn, k);
    const bool tc_form = prm->precision != CS_FP32;
    const bool tex8 = prm->precision == CS_FP8;
    const bool persample = prm->mode == CS_MODE_PERSAMPLE;
    if (tc_form && !tc_supported(k, tex8))
        return cs_set_error(ctx, CS_ERR_UNSUPPORTED,
                            "%s: k=%d too large for the %s tensor-core form", fn, k,
                            tex8 ? "FP8" : "BF16");
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const long long P = (long long)H * W;
    const int S = label_off[n_labels];
    const int Wk = (k + 31) / 32;
    // label offsets and, for the tensor-core form, the first sample tile of each label
    std::vector<int32_t> hoff(2 * (n_labels + 1));
    for (int i = 0; i <= n_labels; ++i) hoff[i] = label_off[i];
    hoff[n_labels + 1] = 0;
    for (int i = 0; i < n_labels; ++i)
        hoff[n_labels + 2 + i] =
            hoff[n_labels + 1 + i] + tc_tiles_per_label(label_off[i + 1] - label_off[i]);
    const int total_tiles = hoff[2 * n_labels + 1];
    const size_t stage_bytes = tc_stage_bytes(k, tex8, persample);

    auto layout = [&](Carve& c, int32_t** d_off, uint32_t** seedbits, int32_t** colbuf,
                      int32_t** vbuf, int32_t** fbuf, int32_t** d2, SampleTables* t) {
        *d_off = c.take<int32_t>(2 * (n_labels + 1));
        *seedbits = c.take<uint32_t>((size_t)n_labels * H * ((W + 31) / 32));
        *colbuf = c.take<int32_t>(P * n_labels);
        *vbuf = c.take<int32_t>(P * n_labels);
        *fbuf = c.take<int32_t>(P * n_labels);
        int32_t* d2s = c.take<int32_t>(dist2 ? 0 : P * n_labels);
        *d2 = dist2 ? dist2 : d2s;
        t->sx = c.take<float>(S);
        t->sy = c.take<float>(S);
        t->sr = c.take<float>(S);
        t->sg = c.take<float>(S);
        t->sb = c.take<float>(S);
        t->sbits = c.take<uint32_t>((size_t)Wk * S);
        t->spop = c.take<int32_t>(S);
        t->rep = c.take<uint32_t>((size_t)n_labels * Wk);
        t->blob = c.take<uint8_t>(tc_form ? (size_t)total_tiles * stage_bytes : 0, 1024);
    };
    int32_t *d_off, *colbuf, *vbuf, *fbuf, *d2;
    uint32_t* seedbits;
    SampleTables t{};
    Carve m(nullptr);
    layout(m, &d_off, &seedbits, &colbuf, &vbuf, &fbuf, &d2, &t);
    s = cs_ensure_scratch(ctx, m.off);
    if (s) return s;
    Carve c(ctx->scratch);
    layout(c, &d_off, &seedbits, &colbuf, &vbuf, &fbuf, &d2, &t);

    cudaError_t e = cudaMemcpyAsync(d_off, hoff.data(), sizeof(int32_t) * hoff.size(),
                                    cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cs_set_error(ctx, CS_ERR_CUDA, "%s: %s", fn, cudaGetErrorString(e));
    EdtArgs ea{H, W, n_labels, d_off, sample_pix, S, seedbits, colbuf, vbuf, fbuf, d2, ctx->d_err};
    {
        StageTimer tm(ctx, CS_STAGE_DIST, st);
        e = launch_edt(ea, st);
    }
    if (e == cudaSuccess) {
        StageTimer tm(ctx, CS_STAGE_GATHER, st);
        e = launch_gather(img, H, W, bitmask, k, n_labels, d_off, sample_pix, S,
                          prm->mode == CS_MODE_FACTORISED, t, st);
    }
    if (e == cudaSuccess) {
        StageTimer tm(ctx, CS_STAGE_SUM, st);
        SumArgs a{};
        a.img = img;
        a.H = H;
        a.W = W;
        a.bitmask = bitmask;
        a.k = k;
        a.Wk = Wk;
        a.n_labels = n_labels;
        a.d_label_off = d_off;
        a.n_samples = S;
        a.t = t;
        a.dist2 = d2;
        a.alpha = (float)prm->alpha;
        a.d_min = (float)prm->d_min;
        a.kappa_beta = (float)prm->kappa_beta;
        a.sigma_c2 = (float)prm->sigma_c2;
        a.mode = prm->mode;
        a.neglog = neglog;
        a.post = post;
        if (!tc_form) {
            e = launch_sum_plain(a, st);
        } else {
            TcLaunch L{};
            L.img = img;
            L.H = H;
            L.W = W;
            L.bitmask = bitmask;
            L.k = k;
            L.n_labels = n_labels;
            L.d_label_off = d_off;
            L.d_tile_off = d_off + n_labels + 1;
            L.total_tiles = total_tiles;
            L.n_samples = S;
            L.t = t;
            L.blob = t.blob;
            L.dist2 = d2;
            L.alpha = a.alpha;
            L.d_min = a.d_min;
            L.kappa_beta = a.kappa_beta;
            L.sigma_c2 = a.sigma_c2;
            L.neglog = neglog;
            L.post = post;
            L.d_err = ctx->d_err;
            L.n_sm = ctx->n_sm;
            L.tex8 = tex8;
            L.persample = persample;
            e = launch_sum_tc(L, st);
        }
    }
    if (e != cudaSuccess) return cs_set_error(ctx, CS_ERR_CUDA, "%s: %s", fn, cudaGetErrorString(e));
    return cs_check_launch(ctx, fn);
}

}  // extern "C"
