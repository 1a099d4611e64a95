// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <string>
#include <vector>

#include "../../include/cosparse.h"

// Device error word layout: err[0] = status code (0 = none), err[1] = detail.
#define CS_DEVERR_GUARD_FULL 101  // co-support guard list overflowed
#define CS_DEVERR_TIMEOUT 102     // bounded wait gave up
#define CS_DEVERR_BAD_SAMPLE 103  // a sample index lies outside the image
#define CS_DEVERR_REFINE_FULL 104 // the FP64 recompute list overflowed

// Largest supported shapes.
#define CS_MAX_K 1024
#define CS_MAX_LABELS 64
#define CS_MAX_CLASSES 16  // colour or texture classes of the unsupervised mode
#define CS_MAX_SIDE 23170  // keeps W^2 + H^2 < 2^31 for the exact distances

struct StageRecord {
    int stage;
    cudaEvent_t beg, end;
};

struct cs_ctx {
    int device = 0;
    std::string err;
    char* scratch = nullptr;
    size_t scratch_cap = 0;
    int* d_err = nullptr;  // 2 ints
    int n_sm = 148;
    // learned surrogate (allocated by the first fit)
    float* surr_buf = nullptr;
    size_t surr_cap = 0;
    int surr_n = 0, surr_nin = 0, surr_set = 0, surr_train = 0, surr_val = 0;
    bool surr_ready = false;
    // per-CTA gradient sums of the network's training kernel
    float* mlp_part = nullptr;
    size_t mlp_part_cap = 0;
    int* last_fb_count = nullptr;  // FP64 recompute count of the last tensor-core sum
    cudaStream_t side = nullptr;   // distance transform overlapping the codes
    cudaStream_t side2 = nullptr;  // sample order overlapping both
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_join2 = nullptr;
    bool profiling = false;
    // timeout-path test hook (cs_test_wait): wait limit of the bounded device
    // waits (0: the kernels' own 1 s) and a one-shot stall of the next
    // solver or tensor-core sum launch
    unsigned long long wait_ns = 0;
    int stall = 0;
    std::vector<StageRecord> records;
    std::vector<cudaEvent_t> event_pool;
    // cs_data_term launch graphs: a call repeated with the same arguments
    // (pointers, sizes, parameters, label offsets) replays the kernels it
    // captured the second time; scratch_gen invalidates them when the scratch
    // moves
    struct DtGraph {
        std::vector<unsigned char> key;
        cudaGraphExec_t exec = nullptr;  // null: seen once, not captured yet
        int* last_fb_count = nullptr;
        unsigned long long used = 0;
    };
    std::vector<DtGraph> dt_graphs;
    unsigned long long dt_clock = 0;
    unsigned scratch_gen = 0;
    cudaStream_t cap = nullptr;  // capture stream of those graphs
};

// Records events around one stage when profiling is on (RAII on the stream).
struct StageTimer {
    cs_ctx* ctx;
    int stage;
    cudaStream_t st;
    cudaEvent_t beg = nullptr, end = nullptr;
    StageTimer(cs_ctx* c, int s, cudaStream_t stream);
    ~StageTimer();
};

// Makes `dev` current for the scope (restores the previous device).
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

// Bump allocator over a context's scratch buffer. First pass with base ==
// nullptr measures the size; the second carves real pointers.
struct Carve {
    char* base;
    size_t off = 0;
    explicit Carve(char* b) : base(b) {}
    template <class T>
    T* take(size_t count, size_t align = 256) {
        off = (off + align - 1) / align * align;
        T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
};

cs_status cs_set_error(cs_ctx* ctx, cs_status code, const char* fmt, ...);
cs_status cs_ensure_scratch(cs_ctx* ctx, size_t bytes);
cs_status cs_check_launch(cs_ctx* ctx, const char* what);

// ---- launchers (each enqueues kernels on `st`; returns cudaError_t) -------

// Patches, codes, co-support bitmasks (FP32 with a rigorous guard band and
// canonical FP64 recomputation of guarded entries).
struct CodesArgs {
    const float* img;
    int H, W;
    const float* omega;
    int k;
    const float* mask;
    int p;
    double tau;
    float* codes;
    float* lead16;
    uint32_t* bitmask;
    // scratch
    float* rownorm;     // k
    int2* guard;        // guard_cap entries
    int guard_cap;
    int* guard_count;   // 1 int
    int* d_err;
    // tensor-core form: operator hi/lo parts in the B-operand layout
    bool tc = false;
    uint8_t* omega_blob = nullptr;
    // patch order 1 (centre, mask, centre again, normalise): every code in
    // double precision in the canonical order (no guard list)
    int order = 0;
};
// FP32 CUDA-core codes, or (a.tc) the tcgen05 split-BF16 GEMM; both followed
// by the canonical FP64 recompute of guarded entries.
cudaError_t launch_codes(const CodesArgs& a, cudaStream_t st);
bool codes_tc_supported(int k, int p);
size_t codes_tc_blob_bytes(int k, int p);
cudaError_t launch_cosupport(const float* codes, long long P, int k, double tau, uint32_t* bitmask,
                             cudaStream_t st);

// Exact squared distance to the nearest scribble of every label.
struct EdtArgs {
    int H, W, n_labels;
    const int32_t* d_label_off;  // device copy, n_labels + 1
    const int32_t* sample_pix;
    int n_samples;
    uint32_t* seedbits;  // scratch n_labels * H * ceil(W/32)
    int32_t* colbuf;  // scratch n_labels * P (horizontal distances)
    int32_t* vbuf;    // scratch n_labels * W * (H + 7) (envelope rows, when not in shared memory)
    int32_t* fbuf;    // scratch, same size (envelope values, likewise)
    int32_t* dist2;   // output n_labels * P
    int* d_err;
};
cudaError_t launch_edt(const EdtArgs& a, cudaStream_t st);

// Smooth co-sparse texture posterior (CS_MODE_SMOOTH), after the Parzen sum.
struct SmoothArgs {
    const float* img;
    int H, W;
    const float* omega;
    int k, p;
    const float* mask;
    const int32_t* sample_pix;
    int S;
    float sigma;
    float* iota_smp;             // scratch k x S (code-major)
    const int32_t* d_label_off;  // device, n_labels + 1
    float* reps;                 // scratch n_labels x k
    int n_labels;
    const int32_t* dist2;
    float alpha, d_min, kappa_beta;
    float* neglog;  // in: -L of the Parzen sum; out: -L with the texture posterior
    float* post;    // optional
};
cudaError_t launch_smooth(const SmoothArgs& a, cudaStream_t st);

// Convex multilabel segmentation (Sec. 4) on a data term.
struct SegArgs {
    const float* f;    // data term, n_labels x H x W
    const float* img;  // H x W x 3
    int H, W, n_labels;
    float lambda, nu, gamma;
    int iterations;
    float* u;          // out: relaxed indicators, n_labels x H x W
    int32_t* labels;   // out (optional): argmax, H x W
    float* scratch;    // seg_scratch_bytes()
    int nblk;          // blocks of the cooperative launch (seg_blocks)
    int* d_err;        // device error word (timeout of a grid barrier)
    unsigned long long wait_ns = 0;  // limit of each grid-barrier wait (0: 1 s)
    bool stall = false;  // timeout-path test: the last block skips its first arrival of
                         // the iterations
};
size_t seg_scratch_bytes(long long P, int n, int nblk);
int seg_blocks(long long P, int n_labels, int n_sm);  // 0 if the kernel cannot be resident
cudaError_t launch_segment(const SegArgs& a, cudaStream_t st);
size_t smooth_smem_bytes(int p, int k, int n_labels);

// Unsupervised mode (Sec. 3.2): iota of every pixel, clusterings, data term.
cudaError_t launch_iota_pixels(const float* img, int H, int W, const float* omega, int k, int p,
                               const float* mask, float sigma, float* iota /* k x H W */,
                               cudaStream_t st);
struct UnsupInit {
    int32_t v[CS_MAX_CLASSES];  // start pixels (validated on the host)
};
struct KmeansArgs {
    const float* X;  // N x 3
    int N, n;
    UnsupInit init;
    int iterations;
    float* C;          // out: n x 3
    int32_t* assign;   // out (optional): N
    void* scratch;     // kmeans_scratch_bytes(n)
    int n_sm;
};
struct KmediansArgs {
    const float* V;  // k x N, code-major
    int N, k, n;
    UnsupInit init;
    int iterations;
    float* C;              // out: n x k
    int32_t* assign;       // out (optional): N
    int32_t* work_assign;  // N (may equal assign)
    int n_sm;
};
struct UnsupFinalArgs {
    const float* img;  // P x 3
    int P;
    const float* V;  // k x P iota
    int k;
    const float* Ccol;
    int nc;
    const float* Ctex;
    int nt;
    float inv2s2, inv_beta;
    float* neglog;     // (nc nt) x P
    int32_t* cassign;  // optional
    int32_t* tassign;  // optional
    int n_sm;
};
size_t kmeans_scratch_bytes(int n);
cudaError_t launch_kmeans(const KmeansArgs& a, cudaStream_t st);
cudaError_t launch_kmedians(const KmediansArgs& a, cudaStream_t st);
cudaError_t launch_unsup_final(const UnsupFinalArgs& a, cudaStream_t st);

// Small host arrays passed by value (no pageable copy, so calls can be
// captured in a CUDA graph): label offsets and first sample tile per label.
struct OffsetsParam {
    int32_t v[2 * (CS_MAX_LABELS + 1)];
};
cudaError_t launch_set_offsets(const OffsetsParam& p, int n, int32_t* dst, cudaStream_t st);

// Per-sample tables (SoA) and the majority co-support of each label.
struct SampleTables {
    float* sx;
    float* sy;
    float* sr;
    float* sg;
    float* sb;
    uint32_t* sbits;  // word-major: [Wk][S]
    int32_t* spop;    // popcount of each sample's bitmask
    uint32_t* rep;    // [n_labels][Wk]
    uint8_t* blob;    // tensor-core sample tiles (ring-stage layout)
    uint32_t* tile_xy;  // tensor-core tile slots: sample position x | y << 16
    int32_t* perm;    // tensor-core sample order (Morton order in chunks of 4096)
};
cudaError_t launch_gather(const float* img, int H, int W, const uint32_t* bitmask, int k,
                          int n_labels, const int32_t* d_label_off, const int32_t* sample_pix,
                          int n_samples, bool want_rep, const SampleTables& t, cudaStream_t st);

// Pixel x sample likelihood sum and label normalisation.
struct SumArgs {
    const float* img;
    int H, W;
    const uint32_t* bitmask;
    int k, Wk;
    int n_labels;
    const int32_t* d_label_off;
    int n_samples;
    SampleTables t;
    const int32_t* dist2;
    float alpha, d_min, kappa_beta;
    float sigma_c2;
    int mode;
    bool rho_var;  // rho is the location kernel's variance (else its standard deviation)
    float* neglog;
    float* post;
    // optional pixel list (device), its length (device) and capacity; with
    // T_out the kernel writes only the log kernel sums T[i][item] (compact)
    const int32_t* pix_list = nullptr;
    const int* list_count = nullptr;
    int list_cap = 0;
    float* T_out = nullptr;
};
cudaError_t launch_sum_plain(const SumArgs& a, cudaStream_t st);

struct TcImage;

// Likelihood-stage plan: shapes, forms and the carved scratch pointers.
struct LikPlan {
    int H, W, k, n_labels, S, total_tiles, n_chunks;
    bool tc_form, tex8, persample;
    size_t stage_bytes;
    OffsetsParam offs;  // label offsets then first sample tile of each label
    int32_t* d_off;
    uint32_t* seedbits;
    int32_t *colbuf, *vbuf, *fbuf, *d2;
    SampleTables t;
    TcImage* desc;  // tensor-core form: descriptor slot
    int4* fb_list;  // tensor-core form: FP64 recompute list (P entries) and count
    int* fb_count;
    float* imax2;   // tensor-core form: per label max |I_j|^2
    unsigned* queue;             // tensor-core form: the sum launch's two claim counters
    unsigned long long* flags;   // tensor-core form: per-pixel flag words
};

typedef LikPlan LikPlanRef;
inline const int32_t* cs_plan_dist2(const LikPlan& L) { return L.d2; }
inline const int32_t* cs_plan_label_off(const LikPlan& L) { return L.d_off; }
inline const uint32_t* cs_plan_rep(const LikPlan& L) { return L.t.rep; }
cs_status cs_check_likelihood_args(cs_ctx* ctx, const char* fn, int H, int W, int k,
                                   int n_labels, const int32_t* label_off, const cs_params* prm);
cs_status cs_plan_likelihood(cs_ctx* ctx, LikPlan& L, int H, int W, int k, int n_labels,
                             const int32_t* label_off, const cs_params* prm, int32_t* dist2,
                             size_t extra, size_t* off_extra);
cudaError_t cs_enqueue_prepare(cs_ctx* ctx, const LikPlan& L, const float* img,
                               const uint32_t* bitmask, const int32_t* sample_pix,
                               const cs_params* prm, cudaStream_t st);
cudaError_t cs_enqueue_exact_list_prepared(cs_ctx* ctx, const LikPlan& L, const float* img,
                                           const uint32_t* bitmask, const cs_params* prm,
                                           const int32_t* list, const int* count, int cap,
                                           float* T_out, float* neglog, float* post,
                                           cudaStream_t st);
cudaError_t cs_enqueue_exact_list(cs_ctx* ctx, const LikPlan& L, const float* img,
                                  const uint32_t* bitmask, const int32_t* sample_pix,
                                  const cs_params* prm, const int32_t* list, const int* count,
                                  int cap, float* T_out, float* neglog, float* post,
                                  cudaStream_t st);

// Tensor-core (tcgen05) pixel x sample sum.
// One image of a sum launch; the launch reads an array of these from device
// memory, in launch order (first_item ascending), and processes items
// (image, pixel tile, label), numbered image by image, pixel tile by pixel
// tile, label by label.
struct TcImage {
    const float* img;
    const uint32_t* bitmask;
    const int32_t* dist2;
    const int32_t* label_off;  // n_labels + 1
    const int32_t* tile_off;   // first sample tile of each label, n_labels + 1
    const uint8_t* blob;       // sample tiles in ring-stage layout
    const uint32_t* tile_xy;   // per tile slot: sample position x | y << 16
    const uint32_t* rep;       // majority co-supports (factorised form)
    float* neglog;
    float* post;
    // per-sample tables (original order), read by the FP64 recompute
    const float *sx, *sy, *sr, *sg, *sb;
    const uint32_t* sbits;  // word-major [Wk][n_samples]
    const float* imax2;     // per label: max_j |I_j|^2 (error bound)
    int n_samples;
    int H, W, ntx, n_labels;
    int n_ptiles;          // pixel tiles of the image
    int first_ptile;       // number of its first pixel tile in the launch
    long long first_item;  // number of the image's first item in the launch
    long long pix_off;     // its first pixel in the launch's flag words
};
struct TcSumParams {
    int k;
    bool tex8, persample;
    float alpha, d_min, kappa_beta, sigma_c2;
    int* d_err;
    int n_sm;
    // pixels with flagged label rows: (image, pixel, label mask low, high),
    // their count (cleared by the launch) and the capacity (>= all pixels)
    int4* fb_list;
    int* fb_count;
    int fb_cap;
    float l_tol;  // relative tolerance on L of the a-priori row bound (0: off)
    bool rho_var;  // rho is the location kernel's variance (else its standard deviation)
    unsigned long long wait_ns = 0;  // limit of each bounded wait (0: the kernel's 1 s)
    bool stall = false;  // timeout-path test: one CTA waits on a barrier nobody completes
    // the launch: items (image, pixel tile, label) and pixels over all
    // images; per image in launch order (HOST) its pixel tiles and labels;
    // the two claim counters (whole pixel tiles, then single items) and the
    // per-pixel flag words (all cleared by the launch)
    long long n_items = 0, total_pixels = 0;
    const int2* shapes = nullptr;  // n_images x (pixel tiles, labels)
    unsigned* queue = nullptr;
    unsigned long long* flags = nullptr;
    // kernel shape: 0 two CTAs per SM where the layout fits, 1 one CTA per SM
    // (16 epilogue warps, deeper sample ring); equal to rounding
    int variant = 0;
};
struct TcLaunch {
    const float* img;
    int H, W;
    const uint32_t* bitmask;
    const int32_t* sample_pix;
    int k;
    int n_labels;
    const int32_t* d_label_off;
    const int32_t* d_tile_off;
    int total_tiles;
    int n_samples;
    SampleTables t;
    uint8_t* blob;
    int n_chunks;  // Morton-sort chunks (4096 samples) over all labels
    const int32_t* dist2;
    float alpha, d_min, kappa_beta, sigma_c2;
    bool rho_var;
    float* neglog;
    float* post;
    int* d_err;
    int n_sm;
    bool tex8;       // texture operands in FP8 (else BF16)
    bool persample;  // per-sample texture kernel (else factorised)
    TcImage* desc;   // device slot receiving this image's descriptor
    // its place in the sum launch: number of its first item and of its first
    // pixel tile, first pixel in the launch's flag words
    long long first_item, pix_off;
    int first_ptile;
    int4* fb_list;   // FP64 recompute list (H W entries) and its count
    int* fb_count;
    unsigned* queue;             // the launch's two claim counters
    unsigned long long* flags;   // flag words (one per pixel)
    float* imax2;    // per label max |I_j|^2 (written by the preparation)
    float l_tol;
    unsigned long long wait_ns;  // as TcSumParams
    bool stall;
};
size_t tc_copy_bytes(int k, bool tex8, bool persample);
int tc_tiles_per_label(int m);
int tc_tile_samples();  // samples per tensor-core sample tile
int tc_pixel_tiles(int H, int W);
bool tc_supported(int k, bool tex8);
// Morton order of the samples (needs only the label offsets and sample
// pixels), then the sample tiles (needs the gathered tables; writes *L.desc),
// or both.
cudaError_t launch_tc_sort(const TcLaunch& L, cudaStream_t st);
cudaError_t launch_tc_tiles(const TcLaunch& L, cudaStream_t st);
cudaError_t launch_tc_prepare(const TcLaunch& L, cudaStream_t st);
// One persistent launch over the items of n_images prepared images (sizes,
// counters and flag words in p).
// CTAs per SM, sample-ring stages, pixel-tile texture buffers and epilogue
// warps of the sum kernel for (k, form, variant); false if unsupported
bool tc_sum_shape(int k, bool tex8, bool persample, int variant, int* shape);
cudaError_t launch_tc_sum(const TcImage* descs, int n_images, const TcSumParams& p,
                          cudaStream_t st);
// For a single image (L.desc must be set): the preparation (Morton sort and
// tile build, or the tile build alone when `sorted`), which needs the
// gathered sample tables but not the distances, then the sum.
cudaError_t launch_sum_tc_prepare(const TcLaunch& L, bool sorted, cudaStream_t st);
cudaError_t launch_sum_tc_run(const TcLaunch& L, cudaStream_t st);

// Validation and planning helpers shared by the entry points.
cs_status cs_check_image(cs_ctx* ctx, const char* fn, int H, int W, int k);
cs_status cs_check_patch(cs_ctx* ctx, const char* fn, const cs_params* prm);
cs_status cs_check_labels(cs_ctx* ctx, const char* fn, int n_labels, const int32_t* label_off);
cs_status cs_check_params(cs_ctx* ctx, const char* fn, const cs_params* prm, int k,
                          bool allow_smooth = false);
void cs_plan_codes(Carve& c, CodesArgs& a, long long P, int k, bool own_bitmask);
bool cs_codes_use_tc(const cs_params* prm, int k);
cs_status cs_check_codes_form(cs_ctx* ctx, const char* fn, const cs_params* prm, int k);
void cs_lik_plan(LikPlan& L, int H, int W, int k, int n_labels, const int32_t* label_off,
                        const cs_params* prm);
void cs_lik_carve(Carve& c, LikPlan& L, int32_t* dist2);
SumArgs cs_sum_args(const LikPlan& L, const float* img, const uint32_t* bitmask,
                    const cs_params* prm, float* neglog, float* post);
TcLaunch cs_tc_launch(cs_ctx* ctx, const LikPlan& L, const float* img, const uint32_t* bitmask,
                      const int32_t* sample_pix, const cs_params* prm, float* neglog,
                      float* post);

// Learned surrogate (MLP) kernels (k_mlp.cu).
int mlp_param_count(int nin, int n);
int mlp_train_ctas(int batch, int n_sm);   // CTAs of one training step
int mlp_part_stride(int nin, int n);       // floats per CTA in the partials buffer
size_t mlp_image_bytes(int nin, int n);    // the kernels' weight image (16-byte multiple)
// the weight image of fp32 parameters (bf16 tiles in the kernels' layout + biases)
cudaError_t launch_mlp_pack(const float* params, int nin, int n, unsigned char* image,
                            cudaStream_t st);
cudaError_t launch_mlp_train(const unsigned char* image, int nin, int n, const float* X,
                             const float* T, int n_rows, long long start, int batch, float* part,
                             int G, int* d_err, uint64_t wait_ns, cudaStream_t st);
// sums G CTAs' partials into g_out (may be NULL) and *loss (may be NULL); with
// m non-NULL also an Adam step (step number t >= 1) on p, rewriting the image
// (when non-NULL) from the updated parameters
cudaError_t launch_reduce_adam(const float* part, int G, int nin, int n, float* p, float* g_out,
                               float* m, float* v, float lr, int t, float* loss,
                               unsigned char* image, cudaStream_t st);
cudaError_t launch_mlp_forward(const unsigned char* image, int nin, int n, const float* X,
                               int rows, float* Z, int n_sm, int* d_err, uint64_t wait_ns,
                               cudaStream_t st);
cudaError_t launch_features(const float* img, const float* lead16, const int32_t* dist2, int H,
                            int W, int n, int feature_set, float d_min, int nin,
                            const int32_t* list, int rows, float* X, cudaStream_t st);
cudaError_t launch_stats(const float* X, int nin, const float* T, int n, int cap, int n_rows,
                         float* stats, cudaStream_t st);
cudaError_t launch_standardize(float* X, int nin, const float* T, int n, int cap, int rows,
                               const float* stats, float* Ts, cudaStream_t st);
cudaError_t launch_init_params(float* p, float* m, float* v, int nin, int n, uint64_t seed,
                               cudaStream_t st);
cudaError_t launch_calib(const float* Z, const float* Ts, int nin, int n, int rows,
                         const float* stats, float* eta, cudaStream_t st);
struct SurrogateEvalArgs {
    const unsigned char* image;  // weight image (launch_mlp_pack)
    int nin, n, feature_set;
    const float* stats;
    const float* eta;
    const float* img;
    const float* lead16;
    int H, W;
    const int32_t* dist2;
    const int32_t* label_off;
    const uint32_t* bitmask;
    const uint32_t* rep;
    int Wk, mode, rule;
    float alpha, d_min, kappa_beta, sigma_c2, margin, eps;
    bool rho_var;
    float* neglog;
    float* post;
    int32_t* fb_list;
    int* fb_count;
    int n_sm;
    int* d_err;
    uint64_t wait_ns;
};
cudaError_t launch_surrogate_eval(const SurrogateEvalArgs& a, cudaStream_t st);
