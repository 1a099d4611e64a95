/*
 * cosparse.h - C ABI of the GB300 (sm_103a) co-sparse data-term library.
 *
 * The library computes the data term of "Co-Sparse Textural Similarity for
 * Image Segmentation" (Nieuwenhuis, Hawe, Kleinsteuber, Cremers): for an RGB
 * image, an analysis operator O, and scribble samples per label, the
 * negative log-likelihood f_i(x) = -log P(I(x), s_x, x | l(x) = i) that the
 * convex multilabel solver of Sec. 4 consumes (Eq. energy1).
 *
 * Conventions shared by every call
 *  - Pointers marked DEVICE must point to memory on the context's device;
 *    pointers marked HOST to ordinary (optionally pinned) host memory.
 *  - The caller owns every input and output buffer. The context owns only
 *    its scratch memory, the device error word and (for the surrogate) the
 *    network weights.
 *  - Buffers are dense, C-contiguous, row-major; pixel index = y * W + x.
 *    Images are H x W x 3 float32 (RGB interleaved, HWC).
 *  - Calls validate their arguments on the host first and return
 *    CS_ERR_INVALID_ARG (or CS_ERR_UNSUPPORTED) before launching anything.
 *    Otherwise the work is enqueued on `stream` (a cudaStream_t, NULL = the
 *    legacy default stream) and the call returns without waiting, except
 *    where a call says it synchronises.
 *  - Errors detected on the device (a bounded wait that gave up, a full
 *    guard list) are recorded in the context's device error word; read it
 *    with cs_sync_status().
 *  - No call throws, exits or aborts. cs_last_error() describes the most
 *    recent failure on the context.
 *  - One context may be used from one host thread at a time, and its calls
 *    must be ordered on one stream: they share the context's scratch memory.
 */
#ifndef COSPARSE_H
#define COSPARSE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int cs_status;
#define CS_OK 0
#define CS_ERR_INVALID_ARG 1 /* bad shape, null pointer, empty label, ... */
#define CS_ERR_CUDA 2        /* a CUDA runtime call failed */
#define CS_ERR_NOMEM 3       /* scratch allocation failed */
#define CS_ERR_TIMEOUT 4     /* a bounded device-side wait gave up */
#define CS_ERR_UNSUPPORTED 5 /* valid but not implemented (e.g. patch side 13) */
#define CS_ERR_DEVICE 6      /* the device error word was set */

/* Likelihood forms (Sec. 3.1). */
#define CS_MODE_PERSAMPLE 0  /* each sample carries k_rho * k_sigma * exp(-TSM/beta) */
#define CS_MODE_FACTORISED 1 /* Eq. (joined): Parzen sum times the Eq. (post_text) softmax */
#define CS_MODE_SMOOTH 2     /* as CS_MODE_FACTORISED with the smooth co-support of Eq. (map_tsm):
                                representatives c_i = elementwise median of iota(O s) over each
                                label's samples (Eq. approx_cosupp), softmax of
                                -||c_i - iota(O s_x)||_1 / beta_i(x); cs_data_term only */

/* Arithmetic forms. */
#define CS_FP32 0 /* CUDA-core FP32 with exact integer distances and popc TSM */
#define CS_BF16 1 /* tensor-core (tcgen05) TSM, colour and location dot products, FP32 accumulation */
#define CS_FP8 2  /* as CS_BF16 with FP8 operands where they are exact */

/* Forms of the operator product (codes). */
#define CS_CODES_AUTO 0 /* tensor cores when supported (k <= 256), else FP32 */
#define CS_CODES_FP32 1 /* CUDA-core FP32 dot products */
#define CS_CODES_TC 2   /* tcgen05 GEMM, split-BF16 operands, FP32 accumulation */

typedef struct cs_ctx cs_ctx;

/*
 * Scalar parameters. Fill with cs_params_default() and override fields.
 *   p          patch side, odd, 3..9 (n = p*p window elements; Sec. 5 uses 9)
 *   mode       CS_MODE_PERSAMPLE, CS_MODE_FACTORISED or CS_MODE_SMOOTH (the
 *              last through cs_data_term only; elsewhere CS_ERR_UNSUPPORTED)
 *   precision  CS_FP32, CS_BF16 or CS_FP8 (the pixel x sample sum)
 *   codes_form the operator product (Sec. 2, a = O s): CS_CODES_AUTO (the
 *              tensor-core form when k <= 256, else FP32), CS_CODES_FP32
 *              (CUDA cores) or CS_CODES_TC (tcgen05 GEMM over three-piece
 *              BF16 splits of O and s, FP32 accumulation). Co-support
 *              bitmasks are bit-exact in every form (guard band + canonical
 *              FP64); the codes returned by cs_codes are within a few 1e-6
 *              |O_j| of the exact values in either form.
 *   tau        co-support threshold: j is in Co(a) iff |a_j| <= tau, the
 *              practical "close to zero" of Sec. 2 (default 0.1)
 *   sigma_c2   variance of the Gaussian colour kernel per channel (Sec. 3.1: 1.3)
 *   alpha      rho_i(x) = alpha * max(|x - x_v|, d_min)  (Sec. 3.1: alpha = 1.3)
 *   d_min      floor on the nearest-scribble distance in pixels (default 1)
 *   kappa_beta beta_i(x) = kappa_beta * rho_i(x): beta proportional to rho (Sec. 3.1)
 *   l_tol      tensor-core forms: a label row whose a-priori error bound on L
 *              exceeds l_tol * max(|L|, 1) is recomputed in FP64 on the GPU
 *              (default 1e-3; 0 recomputes only rows below the FP32 floor;
 *              smaller values recompute more rows, at FP64 speed)
 *   iota_sigma sigma of Eq. (map_tsm), iota(a)_j = exp(-a_j^2 / sigma), for
 *              CS_MODE_SMOOTH (default 0.01, the paper's value; > 0). Its codes
 *              are FP32 dot products of the FP32-normalised patch; a patch
 *              whose centred norm is within the FP32 rounding bound of zero
 *              is taken as flat (every code 0).
 *   rho_variance how rho_i(x) enters the location kernel k_rho (Sec. 3.1
 *              calls rho the kernel's variance but defines it as a length):
 *              0 (default) rho is the standard deviation,
 *              k_rho(u) = exp(-|u|^2 / (2 rho^2)) / (2 pi rho^2);
 *              1 rho is the variance, k_rho(u) = exp(-|u|^2 / (2 rho)) / (2 pi rho).
 *              beta = kappa_beta rho either way. Every likelihood form.
 *   patch_order order of the patch steps (Sec. 3.1 masks "prior to
 *              normalization"): 0 (default) mask, centre, normalise;
 *              1 centre the gray values, mask, centre again, normalise
 *              (bias-invariant). Order 1 computes every code in double
 *              precision in the canonical index order (codes_form is
 *              ignored; the bitmasks are exact, the codes the double values
 *              rounded to FP32); CS_ERR_UNSUPPORTED in CS_MODE_SMOOTH and
 *              cs_unsup_data_term, whose patches are mask-first.
 */
typedef struct {
    int32_t p;
    int32_t mode;
    int32_t precision;
    int32_t codes_form;
    double tau;
    double sigma_c2;
    double alpha;
    double d_min;
    double kappa_beta;
    double l_tol;
    double iota_sigma;
    int32_t rho_variance;
    int32_t patch_order;
} cs_params;

void cs_params_default(cs_params* out);

/* Library version string (static storage). */
const char* cs_version(void);

/*
 * Create a context on CUDA device `device`. *out receives the context; the
 * caller releases it with cs_destroy(). Allocates only the device error
 * word; scratch memory is allocated on first use and grows as needed.
 * Errors: CS_ERR_INVALID_ARG (out NULL or no such device), CS_ERR_CUDA.
 */
cs_status cs_create(cs_ctx** out, int device);
void cs_destroy(cs_ctx* ctx);

/* Message of the last failure on ctx ("" if none). Valid until the next call. */
const char* cs_last_error(const cs_ctx* ctx);

/*
 * Wait for `stream`, then read and clear the device error word.
 * Returns CS_OK, CS_ERR_DEVICE / CS_ERR_TIMEOUT (message in cs_last_error),
 * or CS_ERR_CUDA if the stream reported a CUDA error. Synchronises.
 */
cs_status cs_sync_status(cs_ctx* ctx, void* stream);

/*
 * Test hook for the timeout path of the bounded device waits (the paper has
 * no counterpart: every barrier wait in the library's kernels gives up after
 * a time limit, records a timeout in the device error word and lets the
 * launch end, and this hook lets a test make one such wait run out).
 *   limit_ns  time limit of every bounded wait of the context's later
 *             launches (0 restores the default, 1 s)
 *   stall     one-shot stall of the next launch of one kernel:
 *             CS_STALL_NONE     none (disarms a pending stall)
 *             CS_STALL_SEGMENT  cs_segment: the last block of the cooperative
 *                               launch skips its arrival at the first grid
 *                               barrier of the iterations (needs iterations > 0)
 *             CS_STALL_SUM      the tensor-core sum (cs_likelihood or
 *                               cs_data_term with CS_BF16 / CS_FP8): the
 *                               MMA-issuing thread of the last CTA waits,
 *                               before it issues anything, on a barrier that
 *                               nothing completes
 * The other waits of that launch then run out after limit_ns (or see the
 * abort flag the first one raised); the launch ends, cs_sync_status returns
 * CS_ERR_TIMEOUT, the stalled launch's outputs are undefined, and the
 * context stays usable: the next launch runs normally.
 * Errors: CS_ERR_INVALID_ARG (ctx NULL, limit_ns < 0, unknown stall).
 */
#define CS_STALL_NONE 0
#define CS_STALL_SEGMENT 1
#define CS_STALL_SUM 2
cs_status cs_test_wait(cs_ctx* ctx, int64_t limit_ns, int stall);

/*
 * Patches, codes and co-support bitmasks for every pixel
 * (Sec. 2: a = O s with s a zero-mean, unit-norm patch; Sec. 3.1: gray
 * patch centred at x, multiplied element-wise by a Gaussian mask before the
 * normalisation; Eq. 1: Co(a) = {j : a_j = 0}, read as |a_j| <= tau).
 *
 *   img     DEVICE H x W x 3 float32
 *   omega   DEVICE k x n float32, row-major, n = p*p, window order t = dy*p + dx
 *   mask    DEVICE n float32 (Gaussian weights)
 *   codes   DEVICE P x k float32 or NULL          (P = H*W)
 *   lead16  DEVICE P x 16 float32 or NULL (the first min(k,16) codes, 0-padded)
 *   bitmask DEVICE P x ceil(k/32) uint32 or NULL: bit j of word j>>5 set iff
 *           |a_j| <= tau; pad bits are 0.
 *
 * Patch rule: window pixels clamp to the image edge; gray = 0.299 R +
 * 0.587 G + 0.114 B; v = mask * gray; s = (v - mean v) / ||v - mean v||, or
 * s = 0 when v is constant. Bitmasks are bit-exact against this rule in
 * double precision with sums taken in index order: entries whose FP32 value
 * lies within a rigorous error bound of tau are recomputed that way on the
 * device. `codes` and `lead16` carry the FP32 values.
 * Errors: CS_ERR_INVALID_ARG (H, W < 1; k < 1 or k > 1024; null required
 * pointer), CS_ERR_UNSUPPORTED (p not in 3..9 odd), CS_ERR_NOMEM, CS_ERR_CUDA.
 */
cs_status cs_codes(cs_ctx* ctx, const float* img, int H, int W, const float* omega, int k,
                   const float* mask, const cs_params* prm, float* codes, float* lead16,
                   uint32_t* bitmask, void* stream);

/*
 * cs_codes_noalloc: what cs_codes computes, for callers that cannot allocate
 * device memory. The paper has no counterpart; this exists for callers such
 * as code running while a CUDA graph is being captured (allocation would
 * break the capture), applications whose device memory is entirely owned by
 * another allocator or a fixed budget, and latency-critical loops where
 * cudaMalloc / cudaFree would synchronise the device.
 *
 * It needs no context and allocates nothing: its scratch (operator row norms,
 * the guard counter and a list of up to 2^20 guarded entries) is a fixed
 * ~8 MB array in device memory that every GPU which loads the library holds
 * until the process exits. The caller passes inputs and outputs as for
 * cs_codes (bitmask required), plus dev_status: DEVICE 2 x int32, cleared by
 * the call and set to {101, n} if n entries needed the exact double-precision
 * recheck and n exceeds the 2^20 the scratch holds (only the first 2^20 are
 * rechecked: the bitmask is then not guaranteed exact). Limits: H * W <= 2^20
 * pixels, k <= 1024; larger requests, and the parameter values cs_codes
 * rejects (patch side, tau, patch_order, codes_form), return
 * CS_ERR_INVALID_ARG or CS_ERR_UNSUPPORTED before anything is launched. It always
 * computes the FP32 CUDA-core form of the codes (the codes cs_codes returns
 * with codes_form = CS_CODES_FP32); codes_form = CS_CODES_TC returns
 * CS_ERR_UNSUPPORTED.
 *
 * The first call on a device looks up the scratch array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * All calls share the one array, which keeps the last call's contents: calls
 * whose work overlaps on the GPU (different streams, or different host
 * threads) race and must be serialised by the caller. Failures are reported
 * through cs_last_error(NULL).
 */
cs_status cs_codes_noalloc(const float* img, int H, int W, const float* omega, int k,
                           const float* mask, const cs_params* prm, float* codes, float* lead16,
                           uint32_t* bitmask, int32_t* dev_status, void* stream);

/*
 * Co-support bitmasks of given codes (Eq. 1): bit j of row q is set iff
 * |codes[q*k + j]| <= tau, compared in double precision.
 *   codes DEVICE P x k float32; bitmask DEVICE P x ceil(k/32) uint32.
 */
cs_status cs_cosupport(cs_ctx* ctx, const float* codes, int P, int k, double tau,
                       uint32_t* bitmask, void* stream);

/*
 * Spatially varying likelihoods for every pixel and label (Sec. 3.1).
 *
 * Per-sample form (CS_MODE_PERSAMPLE):
 *   L_i(x) = log (1/m_i) sum_j k_rho(x - x_ij) k_sigma(I(x) - I_ij)
 *                                exp(-TSM(b_x, b_ij) / beta_i(x))
 * Factorised form (CS_MODE_FACTORISED, Eq. joined = Eq. color x Eq. post_text):
 *   L_i(x) = log (1/m_i) sum_j k_rho k_sigma + log softmax_i(-TSM(b_x, c_i) / beta_i(x))
 * with k_rho(u) = exp(-|u|^2 / (2 rho^2)) / (2 pi rho^2),
 * k_sigma(d) = exp(-|d|^2 / (2 sigma_c2)) / (2 pi sigma_c2)^(3/2),
 * rho_i(x) = alpha * max(sqrt(D_i(x)), d_min), D_i(x) the squared distance
 * to the nearest sample of label i (Sec. 3.1), beta_i = kappa_beta * rho_i,
 * TSM the Hamming distance of co-support bitmasks (Eq. tsm_clean) and c_i
 * the majority co-support of the label's samples (Eq. tex-rep).
 *
 *   img        DEVICE H x W x 3 float32
 *   bitmask    DEVICE P x ceil(k/32) uint32 (from cs_codes)
 *   label_off  HOST   n_labels + 1 int32, CSR offsets into sample_pix;
 *              label_off[0] = 0 and every label needs >= 1 sample
 *   sample_pix DEVICE label_off[n_labels] int32 pixel indices (y*W + x)
 *   dist2      DEVICE n_labels x P int32 or NULL: D_i(x), exact
 *   neglog     DEVICE n_labels x P float32: f_i(x) = -L_i(x) (Eq. energy1)
 *   post       DEVICE n_labels x P float32 or NULL: label posteriors
 *              exp(L_i) / sum_l exp(L_l) under a uniform label prior
 * Errors: CS_ERR_INVALID_ARG (empty label, bad offsets, n_labels < 1 or
 * > 64, null required pointer, non-positive sigma_c2/alpha/d_min/kappa_beta),
 * CS_ERR_UNSUPPORTED (k > 256 with the tensor-core forms), CS_ERR_NOMEM,
 * CS_ERR_CUDA.
 */
cs_status cs_likelihood(cs_ctx* ctx, const float* img, int H, int W, const uint32_t* bitmask,
                        int k, int n_labels, const int32_t* label_off,
                        const int32_t* sample_pix, const cs_params* prm, int32_t* dist2,
                        float* neglog, float* post, void* stream);

/*
 * Precision control of the tensor-core forms (CS_BF16, CS_FP8). Every pair
 * exponent e_j (log2 units) is <= 0, so their sum accumulates 2^(e_j + s)
 * in FP32 with the fixed shift s = 96 - ceil(log2 m_i) and cannot overflow.
 * A label row is summed again on the GPU
 * before the call's work completes when it either totals below m_i 2^-100
 * after the shift (terms may have underflowed) or has an a-priori error
 * bound above l_tol * max(|L|, 1): exponents formed in double precision,
 * their offsets from the row maximum exponentiated in FP32 and accumulated
 * in double (two passes); the pixel's label normalisation is then redone in
 * double. The bound (log2 units)
 * adds 2^-15 C Q for the two-piece BF16 colour splits (C = log2 e /
 * (2 sigma_c2), Q = 2 |I| max_j |I_j| + max_j |I_j|^2),
 * 2^-19 (Bt k + C Q + 8 |nA| |x'|^2 + 2 (|log2 S| + log2 m)) for the tensor
 * core's FP32 accumulation of the colour and location MMAs onto the integer
 * texture sum (Bt = log2 e / beta, nA = -log2 e / (2 rho^2), x' the pixel's
 * offset from the centre of its 16 x 8 tile; the location enters relative
 * to that centre), and 6 u (3 (|log2 S| + log2 m) + 2 |R0 + nA |x'|^2| +
 * shift + 1) for the FP32 epilogue, where the pairs' exponents are averaged
 * with the pairs' shares of the row sum S as weights (R0 = -Bt |b_x| -
 * C |I|^2). cs_refined_count returns how many pixels the last tensor-core
 * cs_likelihood / cs_data_term call on ctx recomputed (0 after the plain
 * form). It synchronises `stream`.
 */
cs_status cs_refined_count(cs_ctx* ctx, int32_t* count, void* stream);

/*
 * Convex multilabel segmentation on a data term (Sec. 4): the relaxation of
 * Eq. (energy1) in Eq. (sets), minimised by the primal-dual iteration of
 * Eq. (algo) -- projected ascent in xi (|xi(x)| <= lambda g(x) / 2) and mu
 * (<= 0), projected descent in m ([0, 1]) and u (the simplex, by Michelot's
 * algorithm), over-relaxation of u and m -- and binarised by argmax.
 * g(x) = exp(-|grad I(x)| / gamma) / (2 gamma) on the 8-bit scale (255 I),
 * forward differences; step sizes 1/2 (xi, mu), 1/5 (u), 1/|Omega| (m);
 * start u = 1/n, m = 1.
 *
 *   f          DEVICE n_labels x H x W float32: data term f_i(x), e.g. the
 *              neglog output of cs_data_term
 *   img        DEVICE H x W x 3 float32 (the edge weight g)
 *   sp         lambda >= 0 (boundary weight), nu >= 0 (MDL label cost, 0 for
 *              supervised segmentation), gamma > 0 (paper: 5), iterations >= 0
 *   u          DEVICE n_labels x H x W float32 out: the relaxed indicators
 *   labels     DEVICE H x W int32 out or NULL: argmax_i u_i(x), the lowest
 *              label on ties
 *   n_labels   1..64;  H W < 2^31
 * Defaults (cs_seg_params_default): lambda 1, nu 0, gamma 5, 300 iterations.
 * Uses the context's scratch (4 n P + P floats). Asynchronous on `stream`:
 * one cooperative launch runs every iteration, with grid barriers between
 * the dual and primal steps. Errors: CS_ERR_INVALID_ARG for null or
 * out-of-range arguments; CS_ERR_CUDA when the launch fails; a grid barrier
 * that waits longer than 1 s ends the launch and is reported as
 * CS_ERR_TIMEOUT by the next cs_sync_status.
 */
typedef struct {
    double lambda;
    double nu;
    double gamma;
    int32_t iterations;
    int32_t reserved;
} cs_seg_params;

void cs_seg_params_default(cs_seg_params* out);
cs_status cs_segment(cs_ctx* ctx, const float* f, const float* img, int H, int W, int n_labels,
                     const cs_seg_params* sp, float* u, int32_t* labels, void* stream);

/*
 * Unsupervised mode (Sec. 3.2): segment classes found without scribbles.
 * k-means on the colour pixels gives colour classes, k-medians on the
 * smooth co-supports iota(O s_x) (Eq. map_tsm) texture classes; every
 * (colour class a, texture class b) pair is a segment i = a n_texture + b,
 * and the MDL label cost nu of cs_segment then removes segments.
 *
 * Both clusterings start from caller-given points (the random draw is the
 * caller's), run `iterations` rounds of assignment then update, and return
 * the assignment to the final centres. Assignments are decided in FP32 with
 * the distance summed in a fixed order and the lower class winning ties, so
 * that results are bit-reproducible; a class that wins no point keeps its
 * centre. Asynchronous on `stream`; device pointers unless marked HOST.
 *
 * cs_kmeans: points X (N x 3 float32, e.g. the image), squared Euclidean
 *   distance ((d0^2 + d1^2) + d2^2) without contraction; a centroid is
 *   float32(S / (cnt 2^24)), S the exact integer sum of rint(2^24 v) over
 *   the members (the exact mean of the values rounded to multiples of
 *   2^-24).
 * cs_kmedians: points are the N columns of V (k x N float32, code-major),
 *   l1 distance summed over j = 0 .. k-1 in turn; a centre is the
 *   elementwise median of its members (for an even count the mean of the two
 *   middle values, (lo + hi) * 0.5 in FP32).
 *   n_classes  1..16;  init HOST n_classes start indices in [0, N)
 *   centres    out: n_classes x 3 (k-means) or n_classes x k (k-medians)
 *   assign     out: N int32 or NULL
 * Errors: CS_ERR_INVALID_ARG (null pointer, N < 1, k outside 1..1024,
 * n_classes outside 1..16, a start index outside [0, N), iterations < 0).
 */
cs_status cs_kmeans(cs_ctx* ctx, const float* X, int N, int n_classes, const int32_t* init,
                    int iterations, float* centres, int32_t* assign, void* stream);
cs_status cs_kmedians(cs_ctx* ctx, const float* V, int N, int k, int n_classes,
                      const int32_t* init, int iterations, float* centres, int32_t* assign,
                      void* stream);

/*
 * cs_unsup_data_term: the unsupervised data term of an image. iota of every
 * pixel from FP32 codes (prm->p, prm->iota_sigma; as CS_MODE_SMOOTH), k-means
 * on the pixels' colours, k-medians on iota, then per pixel
 *   f_{a n_t + b}(x) = -log softmax_a(-|I(x) - mu_a|^2 / (2 sigma_c2))
 *                      -log softmax_b(-||c_b - iota(O s_x)||_1 / beta),
 * the product of a colour and a texture posterior as in Eq. post_text
 * (one beta: there are no scribble locations). Uses prm->p, iota_sigma,
 * sigma_c2; the other cs_params fields are ignored.
 *   img, omega, mask  as for cs_codes; k = rows of omega
 *   colour_init       HOST n_colour pixel indices (start centres)
 *   texture_init      HOST n_texture pixel indices (start centres)
 *   neglog            out: (n_colour n_texture) x H x W float32
 *   colour_centres    out or NULL: n_colour x 3
 *   texture_centres   out or NULL: n_texture x k
 *   colour_assign, texture_assign  out or NULL: H x W int32
 * Uses the context's scratch (k H W floats of iota plus small arrays).
 * Errors: CS_ERR_INVALID_ARG (as cs_kmeans / cs_kmedians; n_colour n_texture
 * > 64; iota_sigma, sigma_c2 or beta not > 0; image checks of cs_codes),
 * CS_ERR_UNSUPPORTED (p not in 3..9 odd), CS_ERR_NOMEM, CS_ERR_CUDA.
 */
typedef struct {
    int32_t n_colour;             /* colour classes (k-means), 1..16 */
    int32_t n_texture;            /* texture classes (k-medians), 1..16 */
    int32_t kmeans_iterations;    /* >= 0 */
    int32_t kmedians_iterations;  /* >= 0 */
    double beta;                  /* texture temperature, > 0 */
} cs_unsup_params;

void cs_unsup_params_default(cs_unsup_params* out); /* 4, 4, 10, 10, beta 1 */
cs_status cs_unsup_data_term(cs_ctx* ctx, const float* img, int H, int W, const float* omega,
                             int k, const float* mask, const cs_params* prm,
                             const cs_unsup_params* up, const int32_t* colour_init,
                             const int32_t* texture_init, float* neglog, float* colour_centres,
                             float* texture_centres, int32_t* colour_assign,
                             int32_t* texture_assign, void* stream);

/*
 * The whole data term in one call: patches, codes and co-support bitmasks of
 * every pixel (as cs_codes) followed by the likelihoods (as cs_likelihood).
 * The scribble distance transform and the tensor-core sample order depend
 * only on the samples; they run on two context-owned streams concurrently
 * with the codes. The sample order is joined (CUDA events) before the
 * tensor-core tile build, the distances only before the sum. Arguments as in cs_codes / cs_likelihood; bitmask
 * (DEVICE P x ceil(k/32) uint32) and dist2 may be NULL, in which case they
 * live in scratch. Capturable in a CUDA graph once a first call has sized
 * the scratch (the call allocates only when the scratch must grow).
 * A call repeated with the same arguments (pointers, sizes, parameters, the
 * label offsets' values, stream aside) replays a CUDA graph of its launches
 * that the context captured at the second such call: one launch call instead
 * of about thirty, with results bit-identical to the launches run one by
 * one. The replay reads the buffers' current contents. The context keeps the
 * eight most recently used argument sets; a scratch that grows drops them.
 * Calls under profiling (cs_profile_enable), with a cs_test_wait hook set,
 * or on a stream the caller is capturing run the launches directly.
 */
cs_status cs_data_term(cs_ctx* ctx, const float* img, int H, int W, const float* omega, int k,
                       const float* mask, int n_labels, const int32_t* label_off,
                       const int32_t* sample_pix, const cs_params* prm, uint32_t* bitmask,
                       int32_t* dist2, float* neglog, float* post, void* stream);

/*
 * Batches of images (the same operator, patch mask and parameters for all;
 * every image with its own size, labels and scribbles).
 *
 * The paper segments one image at a time (Sec. 4-5); a batch is this
 * library's way to fill the GPU with many of them. A batch is planned once
 * (cs_batch_create) and run any number of times (cs_batch_run): each run
 * re-reads the images' and scribbles' current contents from the buffers named
 * at creation and rewrites the outputs, so a serving loop refills the same
 * input buffers and runs again. One run:
 *  - per image, on one of n_streams context-independent streams (round robin
 *    in processing order): exact scribble distances, codes and co-support
 *    bitmasks, sample tables and, for the tensor-core forms, the image's
 *    sample tiles and descriptor;
 *  - tensor-core forms: ONE persistent tcgen05 launch over the work items
 *    (image, 16 x 8 pixel tile, label) of all images, in processing order,
 *    claimed by the CTAs from two device counters (whole pixel tiles while
 *    more than about one per CTA is left, then single items); then the FP64
 *    recompute of flagged rows and the label normalisation (plain FP32
 *    form: one sum launch per image on its stream).
 * Processing order: by decreasing pixel x sample pairs (order 0), so that
 * the persistent launch ends with the cheapest items, or as given (order 1).
 * Results are bit-identical to cs_data_term on each image alone with the
 * sum kernel shape that cs_data_term uses (variant 0, the default); the
 * other shape (variant 1, see cs_batch_config) agrees to rounding.
 */
typedef struct {
    const float* img;          /* DEVICE H x W x 3 float32 */
    int32_t H, W;
    int32_t n_labels;          /* 1 .. 64 */
    int32_t reserved;          /* must be 0 */
    const int32_t* label_off;  /* HOST n_labels + 1, read by cs_batch_create only */
    const int32_t* sample_pix; /* DEVICE label_off[n_labels] int32 pixel indices */
    uint32_t* bitmask;         /* DEVICE P x ceil(k/32) out, or NULL (batch memory) */
    int32_t* dist2;            /* DEVICE n_labels x P out, or NULL (batch memory) */
    float* neglog;             /* DEVICE n_labels x P out, required */
    float* post;               /* DEVICE n_labels x P out, or NULL */
} cs_image;

#define CS_BATCH_GRAPH 1    /* capture the run into a CUDA graph after the first run; replay it */
#define CS_BATCH_AUTOTUNE 2 /* first run times each (sum kernel shape, n_streams, order)
                               candidate (synchronises) */

typedef struct cs_batch cs_batch;

/*
 * Validates every image (as cs_data_term would), sizes and allocates the
 * batch's own device memory (it does not use the context's scratch) and
 * fixes the plan. `images` and every label_off array are copied; the device
 * buffers they name must stay valid until cs_batch_destroy. k, omega, mask
 * and prm as in cs_codes / cs_likelihood. flags: CS_BATCH_GRAPH,
 * CS_BATCH_AUTOTUNE (or 0). A tuned configuration is remembered by the
 * context for batches with the same shapes; with the environment variable
 * CS_TUNE_CACHE naming a file it is also read from / appended to that file.
 * Errors: as cs_data_term for the image at fault (the message names its
 * index), CS_ERR_INVALID_ARG for n_images < 1 or > 4096, CS_ERR_NOMEM.
 */
cs_status cs_batch_create(cs_ctx* ctx, const cs_image* images, int n_images, const float* omega,
                          int k, const float* mask, const cs_params* prm, int flags,
                          cs_batch** out);

/* Enqueues one run of the batch on `stream` (ordered after the stream's prior
 * work; the outputs are complete when the stream reaches this point). The
 * first run with CS_BATCH_AUTOTUNE synchronises. Not reentrant: runs of one
 * batch must be ordered on one stream. */
cs_status cs_batch_run(cs_batch* b, void* stream);

/* The configuration in use: streams, order (0 = by decreasing cost,
 * 1 = given), total pixel x sample pairs per run, the tuned run time in
 * milliseconds (-1 when not tuned), the tensor-core sum kernel's shape
 * variant (0: two CTAs per SM where the layout fits, as cs_likelihood and
 * cs_data_term use; 1: one CTA per SM with 16 epilogue warps and a deeper
 * sample ring; the two associate the compensated sums differently and agree
 * to rounding, each within the l_tol bound) and that shape as 4 ints (CTAs per SM, sample-ring stages,
 * pixel-tile texture buffers, epilogue warps; zeros in the plain FP32 form).
 * Any output pointer may be NULL. */
cs_status cs_batch_config(const cs_batch* b, int32_t* n_streams, int32_t* order, double* pairs,
                          double* tuned_ms, int32_t* sum_variant, int32_t* sum_shape);

/* Sets the configuration (1 <= n_streams <= 8, order 0 or 1, sum_variant 0
 * or 1) instead of tuning it; the next run uses it (and recaptures the graph).
 * Errors: CS_ERR_INVALID_ARG. */
cs_status cs_batch_set_config(cs_batch* b, int n_streams, int order, int sum_variant);

/* Frees the batch (waits for its streams first). NULL is a no-op. */
void cs_batch_destroy(cs_batch* b);

/* The likelihood step alone over a batch (as cs_likelihood per image, with
 * one persistent tensor-core sum over all images in the tensor-core forms):
 * each image's `bitmask` is a required DEVICE INPUT (P x ceil(k/32) uint32,
 * e.g. from cs_codes); the other fields as in cs_batch_create. One-shot:
 * plans, runs on `stream` and frees its memory after the run (synchronises
 * the stream). */
cs_status cs_batch_likelihood(cs_ctx* ctx, const cs_image* images, int n_images, int k,
                              const cs_params* prm, void* stream);

/* One-shot batch: create (no flags), run on `stream`, destroy. The batch
 * memory is freed only after the run completes (the call synchronises the
 * stream). */
cs_status cs_batch_data_term(cs_ctx* ctx, const cs_image* images, int n_images,
                             const float* omega, int k, const float* mask, const cs_params* prm,
                             void* stream);

/*
 * Learned surrogate of the data term (not in the paper: an approximation of
 * the Sec. 3.1 likelihood that the exact sum judges and backs up).
 *
 * An n_in -> 64 -> 64 -> 64 -> n_labels MLP with SiLU activations maps
 * per-pixel features to the log kernel sums
 * T_i(x) = log sum_j k_rho k_sigma [exp(-TSM/beta)] of every label;
 * L_i(x) = T_i - log m_i - log(2 pi rho_i^2) - 1.5 log(2 pi sigma_c2) then
 * uses the exact scribble distance transform (and, in the factorised mode,
 * adds the exact texture log-posterior of Eq. post_text). Every contraction
 * runs on the tensor cores (tcgen05, bf16 weights rounded from fp32 masters,
 * activations as two bf16 pieces, fp32 accumulation). Feature sets:
 *   CS_SURR_BASIC     n_in = 21: [R, G, B, x/W, y/H, a_1..a_16] (a = the
 *                     leading codes, cs_codes' lead16)
 *   CS_SURR_EXTENDED  n_in = 45 + n_labels (n_labels <= 19): the basic
 *                     features, log max(d_i, d_min) for every label i (d_i =
 *                     the exact distance to label i's nearest scribble) and
 *                     sin, cos of 2^f pi x/W and of 2^f pi y/H, f = 0..5
 *
 * cs_surrogate_fit: selects training pixels q with u(q) < frac and
 *   validation pixels with frac <= u(q) < frac + min(0.01, 20000/P), where
 *   u(q) = splitmix64(seed ^ q) / 2^64; computes their exact T (FP32 form);
 *   standardises features and targets; trains `steps` Adam steps (minibatch
 *   128 x min(SM count, training rows / 128), learning rate 4e-3 with cosine
 *   decay to 1e-4) with the library's own forward/backward kernels; records
 *   the largest validation error eta of L. The network lives in the
 *   context. Inputs as in cs_likelihood plus lead16 (DEVICE P x 16 float32)
 *   and `features` (CS_SURR_BASIC or CS_SURR_EXTENDED). Asynchronous, but the
 *   pixel selection runs on the host before the call returns.
 * cs_surrogate_eval: evaluates the network at every pixel and writes
 *   neglog/post there, except at the pixels that `rule` sends to the exact
 *   FP32 sum (margin in [0, 1]):
 *     CS_FALLBACK_GUARANTEED  the network's top-2 posterior margin is below
 *                             `margin`, or its top-2 log-likelihood gap is
 *                             below 2.2 eta + log((n_labels - 1) / 0.005)
 *                             (every answered pixel then has max posterior
 *                             error <= 0.005 if all its logits are within
 *                             eta of the exact ones)
 *     CS_FALLBACK_MARGIN      the network's top-2 posterior margin is below
 *                             `margin` (no error guarantee)
 *     CS_FALLBACK_NONE        none: the network answers every pixel
 *   n_fallback (HOST int32, may be NULL) receives their count; when given,
 *   the call synchronises.
 * cs_surrogate_params: copies the fp32 master weights to HOST memory
 *   (layout W1[64][n_in] b1 W2[64][64] b2 W3[64][64] b3 W4[n][64] b4);
 *   *n_params receives their count; host_params may be NULL. Synchronises.
 * cs_mlp_forward / cs_mlp_grad: the network kernels on given DEVICE
 *   parameters (same layout, used rounded to bf16; 1 <= n_in <= 64) and
 *   standardised feature rows X (rows x n_in): outputs Z (rows x n_out), or
 *   the gradient of loss = mean over rows and outputs of (Z - T)^2 / 2 into
 *   grads (DEVICE, cs_mlp_param_count(n_in, n_out) floats) and the loss into
 *   *loss (DEVICE). Weight gradients take the bf16 piece of the activations
 *   (relative error at most 2^-8 of sum |delta| |h| per entry).
 * Errors: CS_ERR_INVALID_ARG (bad sizes, unknown feature set or rule, too
 *   many labels for CS_SURR_EXTENDED, margin outside [0, 1], no fitted
 *   surrogate), CS_ERR_NOMEM,
 *   CS_ERR_CUDA; a device wait that gives up reports CS_ERR_TIMEOUT through
 *   cs_sync_status.
 */
#define CS_SURR_BASIC 0
#define CS_SURR_EXTENDED 1
#define CS_FALLBACK_GUARANTEED 0
#define CS_FALLBACK_MARGIN 1
#define CS_FALLBACK_NONE 2
cs_status cs_surrogate_fit(cs_ctx* ctx, const float* img, int H, int W, const uint32_t* bitmask,
                           const float* lead16, int k, int n_labels, const int32_t* label_off,
                           const int32_t* sample_pix, const cs_params* prm, double frac,
                           int steps, int features, uint64_t seed, void* stream);
cs_status cs_surrogate_eval(cs_ctx* ctx, const float* img, int H, int W, const uint32_t* bitmask,
                            const float* lead16, int k, int n_labels, const int32_t* label_off,
                            const int32_t* sample_pix, const cs_params* prm, int rule,
                            double margin, float* neglog, float* post, int32_t* n_fallback,
                            void* stream);
cs_status cs_surrogate_params(cs_ctx* ctx, float* host_params, int cap, int* n_params);
/*
 * cs_surrogate_info: HOST copies of the standardisation statistics
 * (mu_x[n_in], sd_x[n_in], mu_t[n], sd_t[n]; cap >= 2 n_in + 2n floats, may
 * be NULL), the calibrated validation error eta (nats), the last training
 * step's loss, the training / validation pixel counts and n_in. Synchronises.
 */
cs_status cs_surrogate_info(cs_ctx* ctx, float* host_stats, int cap, float* eta, float* loss,
                            int* n_train, int* n_val, int* n_in);
/*
 * cs_surrogate_save / cs_surrogate_load: the fitted surrogate (FP32 master
 * weights, feature set, standardisation statistics, calibrated eta, last
 * loss, training and validation counts) to / from a file (HOST path; a small
 * versioned binary format, host byte order). Loading replaces the context's
 * surrogate and resets the optimiser state. Both synchronise the device.
 * Errors: CS_ERR_INVALID_ARG (no surrogate to save, unreadable or malformed
 * file), CS_ERR_NOMEM, CS_ERR_CUDA.
 */
cs_status cs_surrogate_save(cs_ctx* ctx, const char* path);
cs_status cs_surrogate_load(cs_ctx* ctx, const char* path);
int cs_mlp_param_count(int n_in, int n_out);
cs_status cs_mlp_forward(cs_ctx* ctx, const float* params, int n_in, int n_out, const float* X,
                         int rows, float* Z, void* stream);
cs_status cs_mlp_grad(cs_ctx* ctx, const float* params, int n_in, int n_out, const float* X,
                      const float* T, int rows, float* grads, float* loss, void* stream);

/*
 * Measured issue rates of the arithmetic pipes the pixel x sample sums use
 * (a measurement aid for their rooflines; the paper has no counterpart):
 * sustained results per SM per clock of ex2.approx (the special-function
 * unit's exponential), popc, FFMA and the packed FFMA2 (fma.rn.f32x2, two
 * results per instruction), from 8 independent chains per thread in one
 * 1024-thread block per SM, each block timed by its SM's cycle counter (so
 * the figures are per clock, whatever the clock frequency was).
 *   out        HOST 4 doubles: ex2, popc, FFMA, FFMA2 results / SM / clock
 *              (median over the SMs)
 *   clock_mhz  HOST double or NULL: the SM clock implied by the slowest
 *              block's cycles over the FFMA launch's event time
 * Allocates a few KB, launches 8 short kernels (about a millisecond each) on
 * the legacy default stream and synchronises the device.
 * Errors: CS_ERR_INVALID_ARG (null ctx or out), CS_ERR_CUDA.
 */
cs_status cs_unit_rates(cs_ctx* ctx, double* out, double* clock_mhz);

/*
 * Stage timing. While enabled, every call records a pair of CUDA events on
 * its stream around each stage it launches:
 *   CS_STAGE_CODES   patches, codes, bitmasks and the FP64 guard pass
 *   CS_STAGE_DIST    exact scribble distance transform
 *   CS_STAGE_GATHER  sample tables and majority co-supports (and, in the
 *                    tensor-core forms, the sample tiles' operand layout)
 *   CS_STAGE_SUM     the pixel x sample likelihood sum and label normalisation
 *   CS_STAGE_SURROGATE  the surrogate network over all pixels
 *   CS_STAGE_TRAIN   the surrogate network's training steps (forward,
 *                    backward, gradient sums and Adam)
 * cs_profile_read waits for the recorded events of `stage`, returns their
 * summed duration in milliseconds and the number of recorded launches, and
 * forgets them. Synchronises on those events only.
 */
#define CS_STAGE_CODES 0
#define CS_STAGE_DIST 1
#define CS_STAGE_GATHER 2
#define CS_STAGE_SUM 3
#define CS_STAGE_SURROGATE 4 /* network evaluation and fallback selection */
#define CS_STAGE_TRAIN 5
#define CS_N_STAGES 6
cs_status cs_profile_enable(cs_ctx* ctx, int on);
cs_status cs_profile_read(cs_ctx* ctx, int stage, double* ms, int* launches);

#ifdef __cplusplus
}
#endif

#endif /* COSPARSE_H */
