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

// Drops every cached data-term graph (they name scratch addresses).
static void drop_dt_graphs(cs_ctx* ctx) {
    for (auto& g : ctx->dt_graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    ctx->dt_graphs.clear();
}

cs_status cs_ensure_scratch(cs_ctx* ctx, size_t bytes) {
    if (bytes <= ctx->scratch_cap) return CS_OK;
    size_t want = bytes + bytes / 4 + (1u << 20);
    drop_dt_graphs(ctx);
    ++ctx->scratch_gen;
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
    out->l_tol = 1e-3;
    out->iota_sigma = 0.01;
    out->rho_variance = 0;
    out->patch_order = 0;
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
        cudaMemset(c->d_err, 0, 2 * sizeof(int)) != cudaSuccess ||
        cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&c->side2, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_join2, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        if (c->d_err) cudaFree(c->d_err);
        if (c->side) cudaStreamDestroy(c->side);
        if (c->side2) cudaStreamDestroy(c->side2);
        if (c->cap) cudaStreamDestroy(c->cap);
        if (c->ev_fork) cudaEventDestroy(c->ev_fork);
        if (c->ev_join) cudaEventDestroy(c->ev_join);
        delete c;
        return cs_set_error(nullptr, CS_ERR_CUDA, "cs_create: cannot set up the context");
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
    if (ctx->surr_buf) cudaFree(ctx->surr_buf);
    if (ctx->mlp_part) cudaFree(ctx->mlp_part);
    if (ctx->side) cudaStreamDestroy(ctx->side);
    if (ctx->side2) cudaStreamDestroy(ctx->side2);
    drop_dt_graphs(ctx);
    if (ctx->cap) cudaStreamDestroy(ctx->cap);
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
    if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
    if (ctx->ev_join2) cudaEventDestroy(ctx->ev_join2);
    delete ctx;
}

const char* cs_last_error(const cs_ctx* ctx) {
    return ctx ? ctx->err.c_str() : g_noctx_err.c_str();
}

void cs_seg_params_default(cs_seg_params* out) {
    if (!out) return;
    memset(out, 0, sizeof *out);
    out->lambda = 1.0;
    out->nu = 0.0;
    out->gamma = 5.0;
    out->iterations = 300;
}

cs_status cs_segment(cs_ctx* ctx, const float* f, const float* img, int H, int W, int n_labels,
                     const cs_seg_params* sp, float* u, int32_t* labels, void* stream) {
    const char* fn = "cs_segment";
    if (!ctx) return cs_set_error(nullptr, CS_ERR_INVALID_ARG, "%s: ctx is NULL", fn);
    if (!f || !img || !sp || !u)
        return cs_set_error(ctx, CS_ERR_INVALID_ARG, "%s: null required pointer", fn);
    if (H < 1 || W < 1 || (long long)H * W > (1ll << 31) - 1)
        return cs_set_error(ctx, CS_ERR_INVALID_ARG, "%s: bad image size %d x %d", fn, H, W);
    if (n_labels < 1 || n_labels > CS_MAX_LABELS)
        return cs_set_error(ctx, CS_ERR_INVALID_ARG, "%s: n_labels=%d outside 1..%d", fn,
                            n_labels, CS_MAX_LABELS);
    if (!(sp->lambda >= 0) || !(sp->nu >= 0) || !(sp->gamma > 0) || sp->iterations < 0)
        return cs_set_error(ctx, CS_ERR_INVALID_ARG,
                            "%s: need lambda >= 0, nu >= 0, gamma > 0, iterations >= 0", fn);
    DeviceGuard g(ctx->device);
    const long long P = (long long)H * W;
    const int nblk = seg_blocks(P, n_labels, ctx->n_sm);
    if (nblk < 1)
        return cs_set_error(ctx, CS_ERR_CUDA, "%s: the solver kernel cannot be resident", fn);
    cs_status s = cs_ensure_scratch(ctx, seg_scratch_bytes(P, n_labels, nblk));
    if (s) return s;
    SegArgs a{f, img, H, W, n_labels, (float)sp->lambda, (float)sp->nu, (float)sp->gamma,
              sp->iterations, u, labels, reinterpret_cast<float*>(ctx->scratch), nblk,
              ctx->d_err};
    a.wait_ns = ctx->wait_ns;
    a.stall = ctx->stall == CS_STALL_SEGMENT;
    if (a.stall) ctx->stall = CS_STALL_NONE;  // one-shot
    cudaError_t e = launch_segment(a, (cudaStream_t)stream);
    if (e != cudaSuccess) return cs_set_error(ctx, CS_ERR_CUDA, "%s: %s", fn, cudaGetErrorString(e));
    return CS_OK;
}

// ---------------------------------------------------------------- unsupervised mode

static cs_status unsup_init(cs_ctx* ctx, const char* fn, const int32_t* init, int n, long long N,
                            UnsupInit* out) {
    if (!init) return cs_set_error(ctx, CS_ERR_INVALID_ARG, "%s: start indices are NULL", fn);
    memset(out, 0, sizeof *out);
    for (int i = 0; i < n; ++i) {
        if (init[i] < 0 || init[i] >= N)
            return cs_set_error(ctx, CS_ERR_INVALID_ARG, "%s: start index %d = %d outside [0, %lld)",
                                fn, i, init[i], N);
        out->v[i] = init[i];
    }
    return CS_OK;
}

static cs_status unsup_classes(cs_ctx* ctx, const char* fn, int n, int iterations) {
    if (n < 1 || n > CS_MAX_CLASSES)
        return cs_set_error(ctx, CS_ERR_INVALID_ARG, "%s: %d classes outside 1..%d", fn, n,
                            CS_MAX_CLASSES);
    if (iterations < 0) return cs_set_error(ctx, CS_ERR_INVALID_ARG, "%s: iterations < 0", fn);
    return CS_OK;
}

cs_status cs_kmeans(cs_ctx* ctx, const float* X, int N, int n_classes, const int32_t* init,
                    int iterations, float* centres, int32_t* assign, void* stream) {
    const char* fn = "cs_kmeans";
    if (!ctx) return cs_set_error(nullptr, CS_ERR_INVALID_ARG, "%s: ctx is NULL", fn);
    if (!X || !centres) return cs_set_error(ctx, CS_ERR_INVALID_ARG, "%s: null pointer", fn);
    if (N < 1) return cs_set_error(ctx, CS_ERR_INVALID_ARG, "%s: N = %d < 1", fn, N);
    cs_status s = unsup_classes(ctx, fn, n_classes, iterations);
    UnsupInit in;
    if (!s) s = unsup_init(ctx, fn, init, n_classes, N, &in);
    if (s) return s;
    DeviceGuard g(ctx->device);
    if ((s = cs_ensure_scratch(ctx, kmeans_scratch_bytes(n_classes)))) return s;
    KmeansArgs a{X, N, n_classes, in, iterations, centres, assign, ctx->scratch, ctx->n_sm};
    cudaError_t e = launch_kmeans(a, (cudaStream_t)stream);
    if (e != cudaSuccess) return cs_set_error(ctx, CS_ERR_CUDA, "%s: %s", fn, cudaGetErrorString(e));
    return CS_OK;
}

cs_status cs_kmedians(cs_ctx* ctx, const float* V, int N, int k, int n_classes,
                      const int32_t* init, int iterations, float* centres, int32_t* assign,
                      void* stream) {
    const char* fn = "cs_kmedians";
    if (!ctx) return cs_set_error(nullptr, CS_ERR_INVALID_ARG, "%s: ctx is NULL", fn);
    if (!V || !centres) return cs_set_error(ctx, CS_ERR_INVALID_ARG, "%s: null pointer", fn);
    if (N < 1 || k < 1 || k > CS_MAX_K)
        return cs_set_error(ctx, CS_ERR_INVALID_ARG, "%s: bad shape N=%d k=%d", fn, N, k);
    cs_status s = unsup_classes(ctx, fn, n_classes, iterations);
    UnsupInit in;
    if (!s) s = unsup_init(ctx, fn, init, n_classes, N, &in);
    if (s) return s;
    DeviceGuard g(ctx->device);
    if (!assign && (s = cs_ensure_scratch(ctx, sizeof(int32_t) * (size_t)N))) return s;
    int32_t* work = assign ? assign : reinterpret_cast<int32_t*>(ctx->scratch);
    KmediansArgs a{V, N, k, n_classes, in, iterations, centres, assign, work, ctx->n_sm};
    cudaError_t e = launch_kmedians(a, (cudaStream_t)stream);
    if (e != cudaSuccess) return cs_set_error(ctx, CS_ERR_CUDA, "%s: %s", fn, cudaGetErrorString(e));
    return CS_OK;
}

void cs_unsup_params_default(cs_unsup_params* out) {
    if (!out) return;
    memset(out, 0, sizeof *out);
    out->n_colour = 4;
    out->n_texture = 4;
    out->kmeans_iterations = 10;
    out->kmedians_iterations = 10;
    out->beta = 1.0;
}

cs_status cs_unsup_data_term(cs_ctx* ctx, const float* img, int H, int W, const float* omega,
                             int k, const float* mask, const cs_params* prm,
                             const cs_unsup_params* up, const int32_t* colour_init,
                             const int32_t* texture_init, float* neglog, float* colour_centres,
                             float* texture_centres, int32_t* colour_assign,
                             int32_t* texture_assign, void* stream) {
    const char* fn = "cs_unsup_data_term";
    if (!ctx) return cs_set_error(nullptr, CS_ERR_INVALID_ARG, "%s: ctx is NULL", fn);
    if (!img || !omega || !mask || !up || !neglog)
        return cs_set_error(ctx, CS_ERR_INVALID_ARG, "%s: null required pointer", fn);
    cs_status s = cs_check_image(ctx, fn, H, W, k);
    if (!s) s = cs_check_patch(ctx, fn, prm);
    if (s) return s;
    if (!(prm->iota_sigma > 0) || !(prm->sigma_c2 > 0) || !(up->beta > 0))
        return cs_set_error(ctx, CS_ERR_INVALID_ARG, "%s: iota_sigma, sigma_c2 and beta must be > 0",
                            fn);
    if (prm->patch_order != 0)
        return cs_set_error(ctx, CS_ERR_UNSUPPORTED, "%s: mask-first patches only", fn);
    const long long P = (long long)H * W;
    UnsupInit ci, ti;
    if (!s) s = unsup_classes(ctx, fn, up->n_colour, up->kmeans_iterations);
    if (!s) s = unsup_classes(ctx, fn, up->n_texture, up->kmedians_iterations);
    if (!s) s = unsup_init(ctx, fn, colour_init, up->n_colour, P, &ci);
    if (!s) s = unsup_init(ctx, fn, texture_init, up->n_texture, P, &ti);
    if (s) return s;
    if (up->n_colour * up->n_texture > CS_MAX_LABELS)
        return cs_set_error(ctx, CS_ERR_INVALID_ARG, "%s: %d x %d segments exceed %d", fn,
                            up->n_colour, up->n_texture, CS_MAX_LABELS);
    DeviceGuard g(ctx->device);
    const int nc = up->n_colour, nt = up->n_texture;
    auto carve = [&](Carve& c, float** iota, float** cc, float** tc, void** km, int32_t** work) {
        *iota = c.take<float>((size_t)k * P);
        *cc = colour_centres ? colour_centres : c.take<float>(3 * (size_t)nc);
        *tc = texture_centres ? texture_centres : c.take<float>((size_t)nt * k);
        *km = c.take<char>(kmeans_scratch_bytes(nc));
        *work = texture_assign ? texture_assign : c.take<int32_t>(P);
    };
    float *iota, *cc, *tc;
    void* km;
    int32_t* work;
    Carve m(nullptr);
    carve(m, &iota, &cc, &tc, &km, &work);
    if ((s = cs_ensure_scratch(ctx, m.off))) return s;
    Carve c(ctx->scratch);
    carve(c, &iota, &cc, &tc, &km, &work);
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = launch_iota_pixels(img, H, W, omega, k, prm->p, mask, (float)prm->iota_sigma,
                                       iota, st);
    if (e == cudaSuccess) {
        KmeansArgs a{img, (int)P, nc, ci, up->kmeans_iterations, cc, nullptr, km, ctx->n_sm};
        e = launch_kmeans(a, st);
    }
    if (e == cudaSuccess) {
        KmediansArgs a{iota, (int)P, k, nt, ti, up->kmedians_iterations, tc, nullptr, work,
                       ctx->n_sm};
        e = launch_kmedians(a, st);
    }
    if (e == cudaSuccess) {
        UnsupFinalArgs a{img, (int)P, iota, k, cc, nc, tc, nt, (float)(0.5 / prm->sigma_c2),
                         (float)(1.0 / up->beta), neglog, colour_assign, texture_assign,
                         ctx->n_sm};
        e = launch_unsup_final(a, st);
    }
    if (e != cudaSuccess) return cs_set_error(ctx, CS_ERR_CUDA, "%s: %s", fn, cudaGetErrorString(e));
    return CS_OK;
}

cs_status cs_refined_count(cs_ctx* ctx, int32_t* count, void* stream) {
    if (!ctx || !count)
        return cs_set_error(ctx, CS_ERR_INVALID_ARG, "cs_refined_count: null argument");
    *count = 0;
    if (!ctx->last_fb_count) return CS_OK;
    DeviceGuard g(ctx->device);
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    int v = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&v, ctx->last_fb_count, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cs_set_error(ctx, CS_ERR_CUDA, "cs_refined_count: %s", cudaGetErrorString(e));
    }
    *count = v;
    return CS_OK;
}

cs_status cs_test_wait(cs_ctx* ctx, int64_t limit_ns, int stall) {
    if (!ctx) return cs_set_error(nullptr, CS_ERR_INVALID_ARG, "cs_test_wait: ctx is NULL");
    if (limit_ns < 0 || (stall != CS_STALL_NONE && stall != CS_STALL_SEGMENT &&
                         stall != CS_STALL_SUM))
        return cs_set_error(ctx, CS_ERR_INVALID_ARG, "cs_test_wait: limit %lld ns, stall %d",
                            (long long)limit_ns, stall);
    ctx->wait_ns = (unsigned long long)limit_ns;
    ctx->stall = stall;
    return CS_OK;
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

}  // extern "C"

// ---------------------------------------------------------------- planning helpers

static int guard_capacity(long long P, int k) {
    long long cap = P * (long long)k / 128 + 65536;
    if (cap > (1ll << 30)) cap = 1ll << 30;
    return (int)cap;
}

cs_status cs_check_image(cs_ctx* ctx, const char* fn, int H, int W, int k) {
    if (H < 1 || W < 1 || H > CS_MAX_SIDE || W > CS_MAX_SIDE)
        return cs_set_error(ctx, CS_ERR_INVALID_ARG, "%s: bad image size %dx%d", fn, W, H);
    if (k < 1 || k > CS_MAX_K)
        return cs_set_error(ctx, CS_ERR_INVALID_ARG, "%s: k=%d outside 1..%d", fn, k, CS_MAX_K);
    return CS_OK;
}

cs_status cs_check_patch(cs_ctx* ctx, const char* fn, const cs_params* prm) {
    if (!prm) return cs_set_error(ctx, CS_ERR_INVALID_ARG, "%s: params is NULL", fn);
    if (prm->p < 1 || (prm->p & 1) == 0)
        return cs_set_error(ctx, CS_ERR_INVALID_ARG, "%s: patch side %d is not odd", fn, prm->p);
    if (prm->p < 3 || prm->p > 9)
        return cs_set_error(ctx, CS_ERR_UNSUPPORTED, "%s: patch side %d not in 3..9", fn, prm->p);
    if (!(prm->tau >= 0.0))
        return cs_set_error(ctx, CS_ERR_INVALID_ARG, "%s: tau must be >= 0", fn);
    if (prm->patch_order != 0 && prm->patch_order != 1)
        return cs_set_error(ctx, CS_ERR_INVALID_ARG, "%s: patch_order must be 0 or 1", fn);
    if (prm->codes_form != CS_CODES_AUTO && prm->codes_form != CS_CODES_FP32 &&
        prm->codes_form != CS_CODES_TC)
        return cs_set_error(ctx, CS_ERR_INVALID_ARG, "%s: unknown codes_form %d", fn,
                            prm->codes_form);
    return CS_OK;
}

bool cs_codes_use_tc(const cs_params* prm, int k) {
    if (prm->codes_form == CS_CODES_FP32 || prm->patch_order == 1) return false;
    return codes_tc_supported(k, prm->p);
}

cs_status cs_check_codes_form(cs_ctx* ctx, const char* fn, const cs_params* prm, int k) {
    if (prm->codes_form == CS_CODES_TC && !codes_tc_supported(k, prm->p))
        return cs_set_error(ctx, CS_ERR_UNSUPPORTED,
                            "%s: the tensor-core codes form supports k <= 256 (k=%d)", fn, k);
    return CS_OK;
}

cs_status cs_check_labels(cs_ctx* ctx, const char* fn, int n_labels,
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

cs_status cs_check_params(cs_ctx* ctx, const char* fn, const cs_params* prm, int k,
                          bool allow_smooth) {
    if (!prm) return cs_set_error(ctx, CS_ERR_INVALID_ARG, "%s: params is NULL", fn);
    if (!(prm->sigma_c2 > 0) || !(prm->alpha > 0) || !(prm->d_min > 0) || !(prm->kappa_beta > 0))
        return cs_set_error(ctx, CS_ERR_INVALID_ARG,
                            "%s: sigma_c2, alpha, d_min and kappa_beta must be > 0", fn);
    if (!(prm->l_tol >= 0.0))
        return cs_set_error(ctx, CS_ERR_INVALID_ARG, "%s: l_tol must be >= 0", fn);
    if (prm->rho_variance != 0 && prm->rho_variance != 1)
        return cs_set_error(ctx, CS_ERR_INVALID_ARG, "%s: rho_variance must be 0 or 1", fn);
    if (prm->mode == CS_MODE_SMOOTH) {
        if (!allow_smooth)
            return cs_set_error(ctx, CS_ERR_UNSUPPORTED,
                                "%s: the smooth texture mode is available through cs_data_term",
                                fn);
        if (!(prm->iota_sigma > 0))
            return cs_set_error(ctx, CS_ERR_INVALID_ARG, "%s: iota_sigma must be > 0", fn);
        if (prm->patch_order != 0)
            return cs_set_error(ctx, CS_ERR_UNSUPPORTED,
                                "%s: the smooth texture mode builds mask-first patches only", fn);
    } else if (prm->mode != CS_MODE_PERSAMPLE && prm->mode != CS_MODE_FACTORISED) {
        return cs_set_error(ctx, CS_ERR_INVALID_ARG, "%s: unknown mode %d", fn, prm->mode);
    }
    if (prm->precision != CS_FP32 && prm->precision != CS_BF16 && prm->precision != CS_FP8)
        return cs_set_error(ctx, CS_ERR_INVALID_ARG, "%s: unknown precision %d", fn,
                            prm->precision);
    if (k > 256)
        return cs_set_error(ctx, CS_ERR_UNSUPPORTED, "%s: k=%d > 256 not supported", fn, k);
    if (prm->precision != CS_FP32 && !tc_supported(k, prm->precision == CS_FP8))
        return cs_set_error(ctx, CS_ERR_UNSUPPORTED,
                            "%s: k=%d too large for the %s tensor-core form", fn, k,
                            prm->precision == CS_FP8 ? "FP8" : "BF16");
    return CS_OK;
}

// Scratch layout of the codes stage.
void cs_plan_codes(Carve& c, CodesArgs& a, long long P, int k, bool own_bitmask) {
    const int cap = guard_capacity(P, k);
    a.rownorm = c.take<float>(k);
    a.guard_count = c.take<int>(1);
    a.guard = c.take<int2>(cap);
    a.guard_cap = cap;
    if (own_bitmask) a.bitmask = c.take<uint32_t>(P * ((k + 31) / 32));
    a.omega_blob = a.tc ? c.take<uint8_t>(codes_tc_blob_bytes(k, a.p), 1024) : nullptr;
}

void cs_lik_plan(LikPlan& L, int H, int W, int k, int n_labels,
                            const int32_t* label_off, const cs_params* prm) {
    L.H = H;
    L.W = W;
    L.k = k;
    L.n_labels = n_labels;
    L.S = label_off[n_labels];
    L.tc_form = prm->precision != CS_FP32;
    L.tex8 = prm->precision == CS_FP8;
    L.persample = prm->mode == CS_MODE_PERSAMPLE;
    for (int i = 0; i <= n_labels; ++i) L.offs.v[i] = label_off[i];
    L.offs.v[n_labels + 1] = 0;
    for (int i = 0; i < n_labels; ++i)
        L.offs.v[n_labels + 2 + i] =
            L.offs.v[n_labels + 1 + i] + tc_tiles_per_label(label_off[i + 1] - label_off[i]);
    L.total_tiles = L.offs.v[2 * n_labels + 1];
    L.n_chunks = 0;
    for (int i = 0; i < n_labels; ++i) L.n_chunks += (label_off[i + 1] - label_off[i] + 4095) / 4096;
    L.stage_bytes = tc_copy_bytes(k, L.tex8, L.persample);
}

void cs_lik_carve(Carve& c, LikPlan& L, int32_t* dist2) {
    const long long P = (long long)L.H * L.W;
    const int n = L.n_labels, S = L.S, Wk = (L.k + 31) / 32;
    L.d_off = c.take<int32_t>(2 * (n + 1));
    L.seedbits = c.take<uint32_t>((size_t)n * L.H * ((L.W + 31) / 32));
    L.colbuf = c.take<int32_t>(P * n);
    // envelope stacks: two halves of (H + 1) / 2 rows per column
    L.vbuf = c.take<int32_t>((size_t)(L.H + 7) * L.W * n);  // S ceil(H / S) <= H + 7 rows
    L.fbuf = c.take<int32_t>((size_t)(L.H + 7) * L.W * n);
    int32_t* d2s = c.take<int32_t>(dist2 ? 0 : P * n);
    L.d2 = dist2 ? dist2 : d2s;
    L.t.sx = c.take<float>(S);
    L.t.sy = c.take<float>(S);
    L.t.sr = c.take<float>(S);
    L.t.sg = c.take<float>(S);
    L.t.sb = c.take<float>(S);
    L.t.sbits = c.take<uint32_t>((size_t)Wk * S);
    L.t.spop = c.take<int32_t>(S);
    L.t.rep = c.take<uint32_t>((size_t)n * Wk);
    L.t.blob = c.take<uint8_t>(L.tc_form ? (size_t)L.total_tiles * L.stage_bytes : 0, 1024);
    L.t.tile_xy = c.take<uint32_t>(L.tc_form ? (size_t)L.total_tiles * tc_tile_samples() : 0);
    L.t.perm = c.take<int32_t>(L.tc_form ? (size_t)S : 0);
    L.desc = c.take<TcImage>(L.tc_form ? 1 : 0);
    L.imax2 = c.take<float>(L.tc_form ? (size_t)n : 0);
    L.fb_list = c.take<int4>(L.tc_form ? (size_t)P : 0);
    L.fb_count = c.take<int>(L.tc_form ? 1 : 0);
    L.queue = c.take<unsigned>(L.tc_form ? 2 : 0);
    L.flags = c.take<unsigned long long>(L.tc_form ? (size_t)P : 0);
}

static cudaError_t enqueue_codes(cs_ctx* ctx, const CodesArgs& a, cudaStream_t st) {
    StageTimer tm(ctx, CS_STAGE_CODES, st);
    return launch_codes(a, st);
}

// Label offsets to the device, then the distance transform, on `st`
// (with_offsets false: the offsets were enqueued earlier on an ordered stream).
static cudaError_t enqueue_distances(cs_ctx* ctx, const LikPlan& L, const int32_t* sample_pix,
                                     cudaStream_t st, bool with_offsets = true) {
    if (with_offsets) {
        cudaError_t e = launch_set_offsets(L.offs, 2 * (L.n_labels + 1), L.d_off, st);
        if (e != cudaSuccess) return e;
    }
    EdtArgs ea{L.H, L.W, L.n_labels, L.d_off, sample_pix, L.S, L.seedbits, L.colbuf,
               L.vbuf, L.fbuf, L.d2, ctx->d_err};
    StageTimer tm(ctx, CS_STAGE_DIST, st);
    return launch_edt(ea, st);
}

SumArgs cs_sum_args(const LikPlan& L, const float* img, const uint32_t* bitmask,
                    const cs_params* prm, float* neglog, float* post) {
    SumArgs a{};
    a.img = img;
    a.H = L.H;
    a.W = L.W;
    a.bitmask = bitmask;
    a.k = L.k;
    a.Wk = (L.k + 31) / 32;
    a.n_labels = L.n_labels;
    a.d_label_off = L.d_off;
    a.n_samples = L.S;
    a.t = L.t;
    a.dist2 = L.d2;
    a.alpha = (float)prm->alpha;
    a.d_min = (float)prm->d_min;
    a.kappa_beta = (float)prm->kappa_beta;
    a.sigma_c2 = (float)prm->sigma_c2;
    a.mode = prm->mode;
    a.rho_var = prm->rho_variance != 0;
    a.neglog = neglog;
    a.post = post;
    return a;
}

TcLaunch cs_tc_launch(cs_ctx* ctx, const LikPlan& L, const float* img, const uint32_t* bitmask,
                      const int32_t* sample_pix, const cs_params* prm, float* neglog,
                      float* post) {
    TcLaunch T{};
    T.img = img;
    T.H = L.H;
    T.W = L.W;
    T.bitmask = bitmask;
    T.sample_pix = sample_pix;
    T.k = L.k;
    T.n_labels = L.n_labels;
    T.d_label_off = L.d_off;
    T.d_tile_off = L.d_off + L.n_labels + 1;
    T.total_tiles = L.total_tiles;
    T.n_samples = L.S;
    T.t = L.t;
    if (prm->mode == CS_MODE_SMOOTH) T.t.rep = nullptr;  // no bitmask texture posterior
    T.blob = L.t.blob;
    T.n_chunks = L.n_chunks;
    T.dist2 = L.d2;
    T.alpha = (float)prm->alpha;
    T.d_min = (float)prm->d_min;
    T.kappa_beta = (float)prm->kappa_beta;
    T.sigma_c2 = (float)prm->sigma_c2;
    T.rho_var = prm->rho_variance != 0;
    T.neglog = neglog;
    T.post = post;
    T.d_err = ctx->d_err;
    T.n_sm = ctx->n_sm;
    T.tex8 = L.tex8;
    T.persample = L.persample;
    T.desc = L.desc;
    T.first_item = 0;
    T.pix_off = 0;
    T.first_ptile = 0;
    T.fb_list = L.fb_list;
    T.fb_count = L.fb_count;
    T.queue = L.queue;
    T.flags = L.flags;
    T.imax2 = L.imax2;
    T.l_tol = (float)prm->l_tol;
    T.wait_ns = ctx->wait_ns;
    T.stall = false;
    return T;
}

// Gather and sum; with `sorted` the tensor-core sample order was already
// enqueued (cs_data_term sorts on a side stream). The gather and the
// tensor-core tile build do not need the distances: with `dist_ready` (the
// distance transform's completion on another stream) the stream waits for
// it only before the sum itself.
static cudaError_t enqueue_sum(cs_ctx* ctx, const LikPlan& L, const float* img,
                               const uint32_t* bitmask, const int32_t* sample_pix,
                               const cs_params* prm, float* neglog, float* post,
                               cudaStream_t st, bool sorted = false,
                               cudaEvent_t dist_ready = nullptr) {
    TcLaunch T{};
    if (L.tc_form) {
        ctx->last_fb_count = L.fb_count;
        T = cs_tc_launch(ctx, L, img, bitmask, sample_pix, prm, neglog, post);
        T.stall = ctx->stall == CS_STALL_SUM;  // the timeout-path test hook, one-shot
        if (T.stall) ctx->stall = CS_STALL_NONE;
    }
    cudaError_t e;
    {
        StageTimer tm(ctx, CS_STAGE_GATHER, st);
        e = launch_gather(img, L.H, L.W, bitmask, L.k, L.n_labels, L.d_off, sample_pix, L.S,
                          !L.persample, L.t, st);
        if (e == cudaSuccess && L.tc_form) e = launch_sum_tc_prepare(T, sorted, st);
    }
    if (e == cudaSuccess && dist_ready) e = cudaStreamWaitEvent(st, dist_ready, 0);
    if (e != cudaSuccess) return e;
    StageTimer tm(ctx, CS_STAGE_SUM, st);
    if (!L.tc_form) return launch_sum_plain(cs_sum_args(L, img, bitmask, prm, neglog, post), st);
    return launch_sum_tc_run(T, st);
}

extern "C" {

// ---------------------------------------------------------------- entry points

cs_status cs_codes(cs_ctx* ctx, const float* img, int H, int W, const float* omega, int k,
                   const float* mask, const cs_params* prm, float* codes, float* lead16,
                   uint32_t* bitmask, void* stream) {
    const char* fn = "cs_codes";
    if (!ctx) return cs_set_error(nullptr, CS_ERR_INVALID_ARG, "%s: ctx is NULL", fn);
    if (!img || !omega || !mask)
        return cs_set_error(ctx, CS_ERR_INVALID_ARG, "%s: null input pointer", fn);
    if (!codes && !lead16 && !bitmask)
        return cs_set_error(ctx, CS_ERR_INVALID_ARG, "%s: no output requested", fn);
    cs_status s = cs_check_image(ctx, fn, H, W, k);
    if (!s) s = cs_check_patch(ctx, fn, prm);
    if (!s) s = cs_check_codes_form(ctx, fn, prm, k);
    if (s) return s;
    DeviceGuard g(ctx->device);
    const long long P = (long long)H * W;
    CodesArgs a{img, H, W, omega, k, mask, prm->p, prm->tau, codes, lead16, bitmask};
    a.tc = cs_codes_use_tc(prm, k);
    a.order = prm->patch_order;
    Carve m(nullptr);
    cs_plan_codes(m, a, P, k, !bitmask);
    if ((s = cs_ensure_scratch(ctx, m.off))) return s;
    Carve c(ctx->scratch);
    cs_plan_codes(c, a, P, k, !bitmask);
    a.d_err = ctx->d_err;
    cudaError_t e = enqueue_codes(ctx, a, (cudaStream_t)stream);
    if (e != cudaSuccess) return cs_set_error(ctx, CS_ERR_CUDA, "%s: %s", fn, cudaGetErrorString(e));
    return cs_check_launch(ctx, fn);
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

}  // extern "C"

// ---------------------------------------------------------------- helpers for other entry points

cs_status cs_check_likelihood_args(cs_ctx* ctx, const char* fn, int H, int W, int k,
                                   int n_labels, const int32_t* label_off, const cs_params* prm) {
    cs_status s = cs_check_image(ctx, fn, H, W, k);
    if (!s) s = cs_check_labels(ctx, fn, n_labels, label_off);
    if (!s) s = cs_check_params(ctx, fn, prm, k);
    return s;
}

// Plans and carves the likelihood scratch with `extra` bytes reserved after
// it (their offset in *off_extra).
cs_status cs_plan_likelihood(cs_ctx* ctx, LikPlan& L, int H, int W, int k, int n_labels,
                             const int32_t* label_off, const cs_params* prm, int32_t* dist2,
                             size_t extra, size_t* off_extra) {
    cs_lik_plan(L, H, W, k, n_labels, label_off, prm);
    Carve m(nullptr);
    cs_lik_carve(m, L, dist2);
    const size_t base = (m.off + 255) / 256 * 256;
    cs_status s = cs_ensure_scratch(ctx, base + extra);
    if (s) return s;
    Carve c(ctx->scratch);
    cs_lik_carve(c, L, dist2);
    *off_extra = base;
    return CS_OK;
}

// distances and sample tables
cudaError_t cs_enqueue_prepare(cs_ctx* ctx, const LikPlan& L, const float* img,
                               const uint32_t* bitmask, const int32_t* sample_pix,
                               const cs_params* prm, cudaStream_t st) {
    cudaError_t e = enqueue_distances(ctx, L, sample_pix, st);
    if (e != cudaSuccess) return e;
    StageTimer tm(ctx, CS_STAGE_GATHER, st);
    return launch_gather(img, L.H, L.W, bitmask, L.k, L.n_labels, L.d_off, sample_pix, L.S,
                         prm->mode == CS_MODE_FACTORISED, L.t, st);
}

// exact plain sum over a device pixel list (after cs_enqueue_prepare): with
// T_out the log kernel sums [n_labels][cap], else neglog/post at the pixels
cudaError_t cs_enqueue_exact_list_prepared(cs_ctx* ctx, const LikPlan& L, const float* img,
                                           const uint32_t* bitmask, const cs_params* prm,
                                           const int32_t* list, const int* count, int cap,
                                           float* T_out, float* neglog, float* post,
                                           cudaStream_t st) {
    SumArgs a = cs_sum_args(L, img, bitmask, prm, neglog, post);
    a.pix_list = list;
    a.list_count = count;
    a.list_cap = cap;
    a.T_out = T_out;
    StageTimer tm(ctx, CS_STAGE_SUM, st);
    return launch_sum_plain(a, st);
}

cudaError_t cs_enqueue_exact_list(cs_ctx* ctx, const LikPlan& L, const float* img,
                                  const uint32_t* bitmask, const int32_t* sample_pix,
                                  const cs_params* prm, const int32_t* list, const int* count,
                                  int cap, float* T_out, float* neglog, float* post,
                                  cudaStream_t st) {
    cudaError_t e = cs_enqueue_prepare(ctx, L, img, bitmask, sample_pix, prm, st);
    if (e != cudaSuccess) return e;
    return cs_enqueue_exact_list_prepared(ctx, L, img, bitmask, prm, list, count, cap, T_out,
                                          neglog, post, st);
}

extern "C" {

cs_status cs_likelihood(cs_ctx* ctx, const float* img, int H, int W, const uint32_t* bitmask,
                        int k, int n_labels, const int32_t* label_off,
                        const int32_t* sample_pix, const cs_params* prm, int32_t* dist2,
                        float* neglog, float* post, void* stream) {
    const char* fn = "cs_likelihood";
    if (!ctx) return cs_set_error(nullptr, CS_ERR_INVALID_ARG, "%s: ctx is NULL", fn);
    if (!img || !bitmask || !sample_pix || !neglog)
        return cs_set_error(ctx, CS_ERR_INVALID_ARG, "%s: null required pointer", fn);
    cs_status s = cs_check_image(ctx, fn, H, W, k);
    if (!s) s = cs_check_labels(ctx, fn, n_labels, label_off);
    if (!s) s = cs_check_params(ctx, fn, prm, k);
    if (s) return s;
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    LikPlan L{};
    cs_lik_plan(L, H, W, k, n_labels, label_off, prm);
    Carve m(nullptr);
    cs_lik_carve(m, L, dist2);
    if ((s = cs_ensure_scratch(ctx, m.off))) return s;
    Carve c(ctx->scratch);
    cs_lik_carve(c, L, dist2);
    cudaError_t e = enqueue_distances(ctx, L, sample_pix, st);
    if (e == cudaSuccess) e = enqueue_sum(ctx, L, img, bitmask, sample_pix, prm, neglog, post, st);
    if (e != cudaSuccess) return cs_set_error(ctx, CS_ERR_CUDA, "%s: %s", fn, cudaGetErrorString(e));
    return cs_check_launch(ctx, fn);
}

cs_status cs_data_term(cs_ctx* ctx, const float* img, int H, int W, const float* omega, int k,
                       const float* mask, int n_labels, const int32_t* label_off,
                       const int32_t* sample_pix, const cs_params* prm, uint32_t* bitmask,
                       int32_t* dist2, float* neglog, float* post, void* stream) {
    const char* fn = "cs_data_term";
    if (!ctx) return cs_set_error(nullptr, CS_ERR_INVALID_ARG, "%s: ctx is NULL", fn);
    if (!img || !omega || !mask || !sample_pix || !neglog)
        return cs_set_error(ctx, CS_ERR_INVALID_ARG, "%s: null required pointer", fn);
    cs_status s = cs_check_image(ctx, fn, H, W, k);
    if (!s) s = cs_check_patch(ctx, fn, prm);
    if (!s) s = cs_check_codes_form(ctx, fn, prm, k);
    if (!s) s = cs_check_labels(ctx, fn, n_labels, label_off);
    if (!s) s = cs_check_params(ctx, fn, prm, k, true);
    if (s) return s;
    const bool smooth = prm->mode == CS_MODE_SMOOTH;
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const long long P = (long long)H * W;
    CodesArgs a{img, H, W, omega, k, mask, prm->p, prm->tau, nullptr, nullptr, bitmask};
    a.tc = cs_codes_use_tc(prm, k);
    a.order = prm->patch_order;
    LikPlan L{};
    cs_lik_plan(L, H, W, k, n_labels, label_off, prm);
    Carve m(nullptr);
    cs_plan_codes(m, a, P, k, !bitmask);
    cs_lik_carve(m, L, dist2);
    if (smooth) {  // smooth texture: sample iota (code-major) and representatives
        m.take<float>((size_t)k * L.S);
        m.take<float>((size_t)n_labels * k);
    }
    if ((s = cs_ensure_scratch(ctx, m.off))) return s;
    Carve c(ctx->scratch);
    cs_plan_codes(c, a, P, k, !bitmask);
    cs_lik_carve(c, L, dist2);
    float* iota_smp = smooth ? c.take<float>((size_t)k * L.S) : nullptr;
    float* reps = smooth ? c.take<float>((size_t)n_labels * k) : nullptr;
    a.d_err = ctx->d_err;
    // every launch of the call on stream st (the caller's, or the capture stream)
    auto enqueue = [&](cudaStream_t st) -> cudaError_t {
        // fork: the distance transform and the tensor-core sample order depend
        // only on the scribbles; they run on the context's two side streams while
        // the codes run on the caller's stream
        cudaError_t e = launch_set_offsets(L.offs, 2 * (L.n_labels + 1), L.d_off, st);
        if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_fork, st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0);
        if (e == cudaSuccess) e = enqueue_distances(ctx, L, sample_pix, ctx->side, false);
        if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_join, ctx->side);
        if (e == cudaSuccess && L.tc_form) {
            e = cudaStreamWaitEvent(ctx->side2, ctx->ev_fork, 0);
            if (e == cudaSuccess)
                e = launch_tc_sort(cs_tc_launch(ctx, L, img, a.bitmask, sample_pix, prm, neglog, post),
                                   ctx->side2);
            if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_join2, ctx->side2);
        }
        if (e == cudaSuccess) e = enqueue_codes(ctx, a, st);
        if (e == cudaSuccess && L.tc_form) e = cudaStreamWaitEvent(st, ctx->ev_join2, 0);
        if (e == cudaSuccess)
            e = enqueue_sum(ctx, L, img, a.bitmask, sample_pix, prm, neglog, post, st, L.tc_form,
                            ctx->ev_join);
        if (e == cudaSuccess && smooth) {
            SmoothArgs sa{img, H, W, omega, k, prm->p, mask, sample_pix, L.S, (float)prm->iota_sigma,
                          iota_smp, L.d_off, reps, n_labels, L.d2, (float)prm->alpha,
                          (float)prm->d_min, (float)prm->kappa_beta, neglog, post};
            e = launch_smooth(sa, st);
        }
        return e;
    };
    cudaError_t e = cudaSuccess;
    // a plain repeated call replays a graph of its launches (one launch call
    // instead of about thirty); not under profiling, the timeout hook, or a
    // capture the caller has open on the stream
    cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
    const bool graphable = !ctx->profiling && ctx->wait_ns == 0 && ctx->stall == 0 &&
                           cudaStreamIsCapturing(st, &cst) == cudaSuccess &&
                           cst == cudaStreamCaptureStatusNone;
    if (!graphable) {
        cudaGetLastError();
        e = enqueue(st);
    } else {
        std::vector<unsigned char> key;
        auto put = [&](const void* v, size_t n) {
            const unsigned char* b = static_cast<const unsigned char*>(v);
            key.insert(key.end(), b, b + n);
        };
        const void* ptrs[] = {img, omega, mask, sample_pix, bitmask, dist2, neglog, post};
        const int ints[] = {H, W, k, n_labels, ctx->device, (int)ctx->scratch_gen};
        put(ptrs, sizeof ptrs);
        put(ints, sizeof ints);
        put(prm, sizeof *prm);
        put(label_off, sizeof(int32_t) * (size_t)(n_labels + 1));
        cs_ctx::DtGraph* hit = nullptr;
        for (auto& gr : ctx->dt_graphs)
            if (gr.key == key) hit = &gr;
        if (!hit) {  // first sight: run directly, remember the key
            if (ctx->dt_graphs.size() >= 8) {  // evict the least recently used
                auto lru = ctx->dt_graphs.begin();
                for (auto it = ctx->dt_graphs.begin(); it != ctx->dt_graphs.end(); ++it)
                    if (it->used < lru->used) lru = it;
                if (lru->exec) cudaGraphExecDestroy(lru->exec);
                ctx->dt_graphs.erase(lru);
            }
            ctx->dt_graphs.push_back(cs_ctx::DtGraph{key, nullptr, nullptr, ++ctx->dt_clock});
            e = enqueue(st);
        } else {
            hit->used = ++ctx->dt_clock;
            if (!hit->exec) {  // second sight: capture on the private stream
                cudaGraph_t graph = nullptr;
                e = cudaStreamBeginCapture(ctx->cap, cudaStreamCaptureModeThreadLocal);
                if (e == cudaSuccess) {
                    const cudaError_t er = enqueue(ctx->cap);
                    e = cudaStreamEndCapture(ctx->cap, &graph);
                    if (er != cudaSuccess) e = er;
                }
                if (e == cudaSuccess) e = cudaGraphInstantiate(&hit->exec, graph, 0);
                if (graph) cudaGraphDestroy(graph);
                hit->last_fb_count = ctx->last_fb_count;
                if (e != cudaSuccess) {  // not capturable here: run directly
                    cudaGetLastError();
                    hit->exec = nullptr;
                    e = enqueue(st);
                }
            }
            if (hit->exec) {
                e = cudaGraphLaunch(hit->exec, st);
                ctx->last_fb_count = hit->last_fb_count;
            }
        }
    }
    if (e != cudaSuccess) return cs_set_error(ctx, CS_ERR_CUDA, "%s: %s", fn, cudaGetErrorString(e));
    return cs_check_launch(ctx, fn);
}

}  // extern "C"
