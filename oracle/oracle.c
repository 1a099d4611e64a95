/*
 * CPU FP64 oracle for the co-sparse data term.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path links, loads or
 * calls this file; only the tests, the smoke check and the CPU baseline leg
 * of the benchmark do. It shares no code with the CUDA library.
 *
 * Every quantity is the paper's definition evaluated literally in double
 * precision, pixel by pixel and sample by sample, with no blocking, fusion
 * or reordering:
 *
 *   patch      Sec. 2 (zero mean, unit norm), Sec. 3.1 (gray patch centred at
 *              x, Gaussian mask applied before the normalisation)
 *   codes      Sec. 2: a = O s
 *   co-support Eq. (1): Co(a) = { j : a_j = 0 }, read as |a_j| <= tau
 *   TSM        Eq. (tsm_clean): Hamming distance of co-support indicators
 *   majority   Eq. (tex-rep): j in Co(z) <=> #{i : j in Co(O s_i)} >= m / 2
 *   distance   Sec. 3.1: rho_i(x) = alpha |x - x_v|, x_v the nearest scribble
 *   Parzen sum Eq. (color): (1/m_i) sum_j k_rho(x - x_ij) k_sigma(I - I_ij)
 *   texture    Eq. (post_text), beta_i proportional to rho_i
 *   data term  Eq. (energy1): f_i = -log P(I(x), s_x, x | l = i)
 *
 * Readings where the paper is silent (each one is a fixed rule here):
 *   gray = (0.299 R + 0.587 G) + 0.114 B; window pixels clamp to the edge;
 *   v = w . g, mu = sum(v)/n, c = v - mu, s = c / sqrt(sum c^2), s = 0 when
 *   sum c^2 == 0; all sums run in index order; the co-support test is
 *   |a_j| <= tau (inclusive); rho = alpha * max(sqrt(D), d_min) is a standard
 *   deviation, k_rho(u) = exp(-|u|^2 / (2 rho^2)) / (2 pi rho^2), or, with
 *   rho_variance = 1, the variance, k_rho(u) = exp(-|u|^2 / (2 rho)) / (2 pi rho)
 *   (Sec. 3.1 calls rho the variance but defines it as a length); the colour
 *   kernel has variance sigma_c2 per channel over d = 3 channels; beta =
 *   kappa_beta * rho; in the per-sample form each sample also carries the
 *   factor exp(-TSM(b_x, b_j) / beta); in the factorised form the texture
 *   factor is the label softmax of Eq. (post_text) against the majority
 *   co-support of each label.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC (no FMA anywhere).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

static double gray_at(const float* img, int W, int y, int x) {
    const float* px = img + ((size_t)y * W + x) * 3;
    double r = (double)px[0], g = (double)px[1], b = (double)px[2];
    return (0.299 * r + 0.587 * g) + 0.114 * b;
}

/* Sec. 2 / Sec. 3.1: masked, zero-mean, unit-norm gray patch at (y, x). */
/* order 0: v = w . g, then centre and normalise (the mask "prior to
 * normalization" of Sec. 3.1 read literally); order 1: centre g first,
 * v = w . (g - mean g), then centre again and normalise. */
static void patch_at(const float* img, int H, int W, int y, int x, const float* mask, int p,
                     int order, double* s) {
    int r = (p - 1) / 2, n = p * p, t;
    double mu = 0.0, ss = 0.0, nrm, mg = 0.0;
    for (int dy = 0; dy < p; ++dy)
        for (int dx = 0; dx < p; ++dx) {
            t = dy * p + dx;
            s[t] = gray_at(img, W, clampi(y + dy - r, 0, H - 1), clampi(x + dx - r, 0, W - 1));
        }
    if (order == 1) {
        for (t = 0; t < n; ++t) mg += s[t];
        mg = mg / (double)n;
        for (t = 0; t < n; ++t) s[t] = (double)mask[t] * (s[t] - mg);
    } else {
        for (t = 0; t < n; ++t) s[t] = (double)mask[t] * s[t];
    }
    for (t = 0; t < n; ++t) mu += s[t];
    mu = mu / (double)n;
    for (t = 0; t < n; ++t) s[t] = s[t] - mu;
    for (t = 0; t < n; ++t) ss += s[t] * s[t];
    if (ss == 0.0) {
        for (t = 0; t < n; ++t) s[t] = 0.0;
        return;
    }
    nrm = sqrt(ss);
    for (t = 0; t < n; ++t) s[t] = s[t] / nrm;
}

/*
 * Codes a = O s and co-support bitmasks for the pixels in pix_list (all P
 * pixels in row-major order when pix_list is NULL). Outputs are indexed by
 * list position: codes[q * k + j], bitmask[q * Wk + (j >> 5)] bit (j & 31).
 */
int oracle_codes(const float* img, int H, int W, const float* omega, int k, const float* mask,
                 int p, double tau, const int32_t* pix_list, int n_pix, double* codes,
                 uint32_t* bitmask, int order) {
    if (H < 1 || W < 1 || p < 1 || (p & 1) == 0 || k < 1 || (order != 0 && order != 1)) return -1;
    int n = p * p, Wk = (k + 31) / 32;
    int count = pix_list ? n_pix : H * W;
#pragma omp parallel for schedule(dynamic, 64)
    for (int q = 0; q < count; ++q) {
        int pix = pix_list ? pix_list[q] : q;
        int y = pix / W, x = pix % W;
        double* s = (double*)malloc(sizeof(double) * (size_t)n);
        patch_at(img, H, W, y, x, mask, p, order, s);
        if (bitmask) memset(bitmask + (size_t)q * Wk, 0, sizeof(uint32_t) * (size_t)Wk);
        for (int j = 0; j < k; ++j) {
            double a = 0.0;
            for (int t = 0; t < n; ++t) a += (double)omega[(size_t)j * n + t] * s[t];
            if (codes) codes[(size_t)q * k + j] = a;
            if (bitmask && fabs(a) <= tau) bitmask[(size_t)q * Wk + (j >> 5)] |= 1u << (j & 31);
        }
        free(s);
    }
    return 0;
}

/* Normalised patches themselves (for the pins on Sec. 2's normalisation). */
int oracle_patches(const float* img, int H, int W, const float* mask, int p,
                   const int32_t* pix_list, int n_pix, double* out, int order) {
    if (H < 1 || W < 1 || p < 1 || (p & 1) == 0 || (order != 0 && order != 1)) return -1;
    int n = p * p, count = pix_list ? n_pix : H * W;
    for (int q = 0; q < count; ++q) {
        int pix = pix_list ? pix_list[q] : q;
        patch_at(img, H, W, pix / W, pix % W, mask, p, order, out + (size_t)q * n);
    }
    return 0;
}

static int bit_of(const uint32_t* b, int j) { return (int)((b[j >> 5] >> (j & 31)) & 1u); }

/* Eq. (tsm_clean): sum over j of |1_Co(a)(j) - 1_Co(b)(j)|, one bit at a time. */
static int tsm_hard(const uint32_t* a, const uint32_t* b, int k) {
    int h = 0;
    for (int j = 0; j < k; ++j) h += abs(bit_of(a, j) - bit_of(b, j));
    return h;
}

int oracle_tsm(const uint32_t* a, const uint32_t* b, int k) { return tsm_hard(a, b, k); }

/* Eq. (tex-rep): bit j of label i's representative is set iff at least half
 * of the label's samples have j in their co-support (2 * count >= m_i). */
int oracle_majority(const uint32_t* bits_smp, int k, int n_labels, const int32_t* label_off,
                    uint32_t* rep) {
    int Wk = (k + 31) / 32;
    for (int i = 0; i < n_labels; ++i) {
        int m = label_off[i + 1] - label_off[i];
        if (m < 1) return -1;
        memset(rep + (size_t)i * Wk, 0, sizeof(uint32_t) * (size_t)Wk);
        for (int j = 0; j < k; ++j) {
            int cnt = 0;
            for (int q = label_off[i]; q < label_off[i + 1]; ++q)
                cnt += bit_of(bits_smp + (size_t)q * Wk, j);
            if (2 * cnt >= m) rep[(size_t)i * Wk + (j >> 5)] |= 1u << (j & 31);
        }
    }
    return 0;
}

/* Sec. 3.1: squared distance from each listed pixel to the nearest scribble
 * sample of each label, by brute force over the label's samples. */
int oracle_dist2(int H, int W, int n_labels, const int32_t* label_off, const int32_t* sample_pix,
                 const int32_t* pix_list, int n_pix, int64_t* dist2) {
    int count = pix_list ? n_pix : H * W;
    for (int i = 0; i < n_labels; ++i)
        if (label_off[i + 1] - label_off[i] < 1) return -1;
#pragma omp parallel for schedule(dynamic, 64)
    for (int q = 0; q < count; ++q) {
        int pix = pix_list ? pix_list[q] : q;
        int64_t y = pix / W, x = pix % W;
        for (int i = 0; i < n_labels; ++i) {
            int64_t best = -1;
            for (int s = label_off[i]; s < label_off[i + 1]; ++s) {
                int64_t sy = sample_pix[s] / W, sx = sample_pix[s] % W;
                int64_t d = (x - sx) * (x - sx) + (y - sy) * (y - sy);
                if (best < 0 || d < best) best = d;
            }
            dist2[(size_t)i * count + q] = best;
        }
    }
    (void)H;
    return 0;
}

/*
 * Log-likelihoods L[i][q] = log P(I(x), s_x, x | l = i), their negatives
 * (the data term f_i of Eq. energy1) and the label posteriors.
 *
 * bits_px:  co-support of each listed pixel (n_pix x Wk)
 * bits_smp: co-support of each scribble sample (n_samples x Wk, CSR order)
 * mode 0:   per-sample product of location, colour and texture kernels
 * mode 1:   factorised, Eq. (joined): Parzen colour-location sum times the
 *           texture softmax of Eq. (post_text) on the majority co-supports
 * mode 2:   the Parzen colour-location sum alone (the smooth texture
 *           posterior of Eq. (post_text) is added by the Python layer)
 * dist2:    optional output, n_labels x n_pix
 */
int oracle_likelihood(const float* img, int H, int W, const uint32_t* bits_px,
                      const uint32_t* bits_smp, int k, int n_labels, const int32_t* label_off,
                      const int32_t* sample_pix, double sigma_c2, double alpha, double d_min,
                      double kappa_beta, int mode, int rho_variance, const int32_t* pix_list,
                      int n_pix, double* L,
                      double* neglog, double* post, int64_t* dist2_out) {
    int Wk = (k + 31) / 32;
    int count = pix_list ? n_pix : H * W;
    if (n_labels < 1 || k < 1 || sigma_c2 <= 0.0 || alpha <= 0.0 || d_min <= 0.0 ||
        kappa_beta <= 0.0 || (mode != 0 && mode != 1 && mode != 2) ||
        (rho_variance != 0 && rho_variance != 1))
        return -1;
    for (int i = 0; i < n_labels; ++i)
        if (label_off[i + 1] - label_off[i] < 1) return -1;
    uint32_t* rep = NULL;
    if (mode == 1) {
        rep = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)n_labels * Wk);
        oracle_majority(bits_smp, k, n_labels, label_off, rep);
    }
    const double log_col_norm = 1.5 * log(2.0 * M_PI * sigma_c2);
#pragma omp parallel for schedule(dynamic, 16)
    for (int q = 0; q < count; ++q) {
        int pix = pix_list ? pix_list[q] : q;
        int64_t y = pix / W, x = pix % W;
        const float* Ix = img + (size_t)pix * 3;
        const uint32_t* bx = bits_px + (size_t)q * Wk;
        double* Lq = (double*)malloc(sizeof(double) * (size_t)n_labels);
        double* Tq = (double*)malloc(sizeof(double) * (size_t)n_labels);
        int mstart, mend;
        for (int i = 0; i < n_labels; ++i) {
            mstart = label_off[i];
            mend = label_off[i + 1];
            /* nearest scribble of label i */
            int64_t D = -1;
            for (int s = mstart; s < mend; ++s) {
                int64_t sy = sample_pix[s] / W, sx = sample_pix[s] % W;
                int64_t d = (x - sx) * (x - sx) + (y - sy) * (y - sy);
                if (D < 0 || d < D) D = d;
            }
            if (dist2_out) dist2_out[(size_t)i * count + q] = D;
            double dist = sqrt((double)D);
            double rho = alpha * (dist > d_min ? dist : d_min);
            double beta = kappa_beta * rho;
            double s2 = rho_variance ? rho : rho * rho; /* variance of the location kernel */
            /* first pass: exponents and their maximum */
            double emax = -INFINITY;
            for (int s = mstart; s < mend; ++s) {
                int64_t sy = sample_pix[s] / W, sx = sample_pix[s] % W;
                double dloc = (double)((x - sx) * (x - sx) + (y - sy) * (y - sy));
                const float* Is = img + (size_t)sample_pix[s] * 3;
                double dc = 0.0;
                for (int c = 0; c < 3; ++c) {
                    double d = (double)Ix[c] - (double)Is[c];
                    dc += d * d;
                }
                double e = -dloc / (2.0 * s2) - dc / (2.0 * sigma_c2);
                if (mode == 0) e -= (double)tsm_hard(bx, bits_smp + (size_t)s * Wk, k) / beta;
                if (e > emax) emax = e;
            }
            /* second pass: sum of exp(e - max) */
            double sum = 0.0;
            for (int s = mstart; s < mend; ++s) {
                int64_t sy = sample_pix[s] / W, sx = sample_pix[s] % W;
                double dloc = (double)((x - sx) * (x - sx) + (y - sy) * (y - sy));
                const float* Is = img + (size_t)sample_pix[s] * 3;
                double dc = 0.0;
                for (int c = 0; c < 3; ++c) {
                    double d = (double)Ix[c] - (double)Is[c];
                    dc += d * d;
                }
                double e = -dloc / (2.0 * s2) - dc / (2.0 * sigma_c2);
                if (mode == 0) e -= (double)tsm_hard(bx, bits_smp + (size_t)s * Wk, k) / beta;
                sum += exp(e - emax);
            }
            double m = (double)(mend - mstart);
            Lq[i] = emax + log(sum) - log(m) - log(2.0 * M_PI * s2) - log_col_norm;
            if (mode == 1) Tq[i] = -(double)tsm_hard(bx, rep + (size_t)i * Wk, k) / beta;
        }
        if (mode == 1) {
            /* Eq. (post_text): texture posterior, softmax over labels */
            double tmax = -INFINITY, ts = 0.0;
            for (int i = 0; i < n_labels; ++i)
                if (Tq[i] > tmax) tmax = Tq[i];
            for (int i = 0; i < n_labels; ++i) ts += exp(Tq[i] - tmax);
            double tlse = tmax + log(ts);
            for (int i = 0; i < n_labels; ++i) Lq[i] += Tq[i] - tlse;
        }
        /* label posteriors under a uniform label prior */
        double lmax = -INFINITY, ls = 0.0;
        for (int i = 0; i < n_labels; ++i)
            if (Lq[i] > lmax) lmax = Lq[i];
        for (int i = 0; i < n_labels; ++i) ls += exp(Lq[i] - lmax);
        double llse = lmax + log(ls);
        for (int i = 0; i < n_labels; ++i) {
            if (L) L[(size_t)i * count + q] = Lq[i];
            if (neglog) neglog[(size_t)i * count + q] = -Lq[i];
            if (post) post[(size_t)i * count + q] = exp(Lq[i] - llse);
        }
        free(Lq);
        free(Tq);
    }
    free(rep);
    (void)H;
    return 0;
}
