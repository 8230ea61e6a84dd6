/*
 * CPU oracle for maximum-Tsallis-entropy threshold selection (Chang & Sheu,
 * "GPU acceleration of a patient-specific airway image segmentation and its
 * assessment", section II-C "Segmentation", subsections "Thresholding" and
 * "Tsallis entropy", and Algorithm 1).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the slow, plainly written reference
 * that the GPU path is checked against. Only the tests, the package's smoke()
 * check and the benchmark's CPU-baseline leg load it; the product path never
 * calls it and shares no code with it.
 *
 * Everything is double precision, with plain loops in the order the paper
 * writes its sums. Histograms are int64 counts.
 *
 * Notation (section II-C, "Tsallis entropy"): p_i are normalised bin
 * probabilities, alpha (q) the Tsallis index, t the threshold on the grey
 * level, s the threshold on the local-mean level, L the number of levels.
 * Class 1 is bins 0..t (and 0..s), class 2 is bins t+1..L-1 (and s+1..L-1).
 *
 * Readings where the paper is silent or garbled:
 *   - bins: b = clamp(v, lo, lo+L-1) - lo (out-of-range values go to the end
 *     bins, as the paper sends -2000 background to level 0);
 *   - a threshold t is valid only when both classes hold mass (P_1 > 0 and
 *     P_2 > 0); otherwise the entropies are 0/0 and t is skipped;
 *   - alpha = 1 is the Shannon (Kapur) limit of the Tsallis form;
 *   - the 2-D mean image uses floor(sum / count) over a 3x3 (single slice) or
 *     3x3x3 (volume) window with clamp-to-edge indexing;
 *   - the argmax takes the smallest t (then s) among equal maxima.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------ histograms */

/* Measurement space of section I "Thresholding" (Fig. 2): counts per level. */
int oracle_hist1d(const int16_t* vol, int64_t n, int32_t lo, int32_t L, int64_t* hist) {
    if (!vol || !hist || n < 0 || L < 2) return 1;
    for (int32_t i = 0; i < L; ++i) hist[i] = 0;
    for (int64_t k = 0; k < n; ++k) {
        int32_t b = (int32_t)vol[k] - lo;
        if (b < 0) b = 0;
        if (b > L - 1) b = L - 1;
        hist[b] += 1;
    }
    return 0;
}

static int64_t clampi(int64_t v, int64_t lo, int64_t hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* Grey level of the 2-D form: the 1-D bin shifted down to L2 levels. */
static int32_t grey_level(int16_t v, int32_t lo, int32_t L1, int32_t shift) {
    int32_t b = (int32_t)v - lo;
    if (b < 0) b = 0;
    if (b > L1 - 1) b = L1 - 1;
    return b >> shift;
}

/*
 * Section II-C "Tsallis entropy": the average image g (3x3 mean, floor of the
 * mean) and the 2-D histogram h(i, j) of (grey level f, mean level g).
 * With nz > 1 the window is 3x3x3 and the divisor 27; with nz == 1 it is 3x3
 * and 9. Counts, not probabilities, are returned: hist[i * L2 + j].
 * If g_out is non-null it receives the grey level f of every voxel and
 * m_out the mean level g.
 */
int oracle_hist2d(const int16_t* vol, int64_t nx, int64_t ny, int64_t nz, int32_t lo, int32_t L1,
                  int32_t shift, int64_t* hist, uint8_t* f_out, uint8_t* m_out) {
    if (!vol || !hist || nx < 1 || ny < 1 || nz < 1 || shift < 0 || shift > 15) return 1;
    int32_t L2 = L1 >> shift;
    if (L2 < 2 || L2 > 256) return 1;
    if (L1 & ((1 << shift) - 1)) return 1; /* grey levels b >> shift must stay below L2 */
    memset(hist, 0, sizeof(int64_t) * (size_t)L2 * (size_t)L2);
    int dz = nz > 1 ? 1 : 0;
    int64_t count = nz > 1 ? 27 : 9;
    for (int64_t z = 0; z < nz; ++z)
        for (int64_t y = 0; y < ny; ++y)
            for (int64_t x = 0; x < nx; ++x) {
                int64_t sum = 0;
                for (int64_t k = -dz; k <= dz; ++k)
                    for (int64_t j = -1; j <= 1; ++j)
                        for (int64_t i = -1; i <= 1; ++i) {
                            int64_t zz = clampi(z + k, 0, nz - 1);
                            int64_t yy = clampi(y + j, 0, ny - 1);
                            int64_t xx = clampi(x + i, 0, nx - 1);
                            sum += grey_level(vol[(zz * ny + yy) * nx + xx], lo, L1, shift);
                        }
                int64_t f = grey_level(vol[(z * ny + y) * nx + x], lo, L1, shift);
                int64_t g = sum / count; /* sum >= 0, so this is the floor */
                hist[f * L2 + g] += 1;
                if (f_out) f_out[(z * ny + y) * nx + x] = (uint8_t)f;
                if (m_out) m_out[(z * ny + y) * nx + x] = (uint8_t)g;
            }
    return 0;
}

/* ------------------------------------------------------------ objective */

/* One class's Tsallis entropy from its probabilities already divided by the
 * class mass: (1 - sum r^alpha) / (alpha - 1); Shannon at alpha == 1. */
static double tsallis_from_sum(double sum_pow, double alpha) { return (1.0 - sum_pow) / (alpha - 1.0); }

/* The objective phi_alpha = H1 + H2 + (1 - alpha) H1 H2 (section II-C). */
static double pseudo_additive(double h1, double h2, double alpha) { return h1 + h2 + (1.0 - alpha) * h1 * h2; }

/*
 * Definition mode, 1-D reading of section II-C: for every t, normalise
 * p_i = h_i / N, form P_1(t) and P_2(t) by summing p, and each class entropy
 * by summing (p_i / P_k)^alpha over its bins, with no prefix sums. O(L^2).
 * phi[t] for t in [0, L-2]; valid[t] = 1 when both classes hold mass.
 */
int oracle_objective1d_def(const int64_t* h, int32_t L, double alpha, double* phi, uint8_t* valid) {
    if (!h || !phi || !valid || L < 2 || !(alpha > 0.0) || !isfinite(alpha)) return 1;
    int64_t N = 0;
    for (int32_t i = 0; i < L; ++i) N += h[i];
    if (N <= 0) {
        for (int32_t t = 0; t < L - 1; ++t) { phi[t] = 0.0; valid[t] = 0; }
        return 0;
    }
    double* p = (double*)malloc(sizeof(double) * (size_t)L);
    if (!p) return 2;
    for (int32_t i = 0; i < L; ++i) p[i] = (double)h[i] / (double)N;
    for (int32_t t = 0; t < L - 1; ++t) {
        double P1 = 0.0, P2 = 0.0;
        int64_t n1 = 0, n2 = 0;
        for (int32_t i = 0; i <= t; ++i) { P1 += p[i]; n1 += h[i]; }
        for (int32_t i = t + 1; i < L; ++i) { P2 += p[i]; n2 += h[i]; }
        if (n1 == 0 || n2 == 0) { phi[t] = 0.0; valid[t] = 0; continue; }
        double H1, H2;
        if (alpha == 1.0) {
            H1 = 0.0; H2 = 0.0;
            for (int32_t i = 0; i <= t; ++i) if (p[i] > 0) { double r = p[i] / P1; H1 -= r * log(r); }
            for (int32_t i = t + 1; i < L; ++i) if (p[i] > 0) { double r = p[i] / P2; H2 -= r * log(r); }
        } else {
            double s1 = 0.0, s2 = 0.0;
            for (int32_t i = 0; i <= t; ++i) s1 += pow(p[i] / P1, alpha);
            for (int32_t i = t + 1; i < L; ++i) s2 += pow(p[i] / P2, alpha);
            H1 = tsallis_from_sum(s1, alpha);
            H2 = tsallis_from_sum(s2, alpha);
        }
        phi[t] = pseudo_additive(H1, H2, alpha);
        valid[t] = 1;
    }
    free(p);
    return 0;
}

/*
 * Plain-prefix mode, written separately: running sums of p_i and p_i^alpha
 * (p_i ln p_i at alpha == 1) from the left for class 1 and from the right for
 * class 2, so sum_{i<=t} (p_i/P_1)^alpha = (sum p_i^alpha) / P_1^alpha.
 * O(L). Same outputs as the definition mode.
 */
int oracle_objective1d_prefix(const int64_t* h, int32_t L, double alpha, double* phi, uint8_t* valid) {
    if (!h || !phi || !valid || L < 2 || !(alpha > 0.0) || !isfinite(alpha)) return 1;
    int64_t N = 0;
    for (int32_t i = 0; i < L; ++i) N += h[i];
    double* P1 = (double*)malloc(sizeof(double) * (size_t)L * 4);
    int64_t* n1 = (int64_t*)malloc(sizeof(int64_t) * (size_t)L * 2);
    if (!P1 || !n1) { free(P1); free(n1); return 2; }
    double* S1 = P1 + L;      /* left running sum of p^alpha (or p ln p) */
    double* P2 = P1 + 2 * L;  /* right running mass, P2[t] = sum_{i>t} p_i */
    double* S2 = P1 + 3 * L;
    int64_t* n2 = n1 + L;
    double accP = 0.0, accS = 0.0;
    int64_t accN = 0;
    for (int32_t i = 0; i < L; ++i) {
        double p = N > 0 ? (double)h[i] / (double)N : 0.0;
        accP += p;
        accN += h[i];
        if (p > 0) accS += alpha == 1.0 ? p * log(p) : pow(p, alpha);
        P1[i] = accP; S1[i] = accS; n1[i] = accN;
    }
    accP = 0.0; accS = 0.0; accN = 0;
    for (int32_t i = L - 1; i >= 0; --i) {
        /* P2[i] holds the sums over bins > i */
        P2[i] = accP; S2[i] = accS; n2[i] = accN;
        double p = N > 0 ? (double)h[i] / (double)N : 0.0;
        accP += p;
        accN += h[i];
        if (p > 0) accS += alpha == 1.0 ? p * log(p) : pow(p, alpha);
    }
    for (int32_t t = 0; t < L - 1; ++t) {
        if (n1[t] == 0 || n2[t] == 0) { phi[t] = 0.0; valid[t] = 0; continue; }
        double H1, H2;
        if (alpha == 1.0) {
            /* -sum (p/P) ln(p/P) = ln P - (sum p ln p) / P */
            H1 = log(P1[t]) - S1[t] / P1[t];
            H2 = log(P2[t]) - S2[t] / P2[t];
        } else {
            H1 = tsallis_from_sum(S1[t] / pow(P1[t], alpha), alpha);
            H2 = tsallis_from_sum(S2[t] / pow(P2[t], alpha), alpha);
        }
        phi[t] = pseudo_additive(H1, H2, alpha);
        valid[t] = 1;
    }
    free(P1);
    free(n1);
    return 0;
}

/*
 * Definition mode of the 2-D form (section II-C): quadrant 1 is
 * {i <= t, j <= s}, quadrant 2 is {i > t, j > s}; the other two quadrants
 * are ignored. P_1(t,s), P_2(t,s) and both entropies are summed directly.
 * O(L^4): for small L only. phi[t * (L-1) + s].
 */
int oracle_objective2d_def(const int64_t* h, int32_t L, double alpha, double* phi, uint8_t* valid) {
    if (!h || !phi || !valid || L < 2 || !(alpha > 0.0) || !isfinite(alpha)) return 1;
    int64_t N = 0;
    for (int64_t k = 0; k < (int64_t)L * L; ++k) N += h[k];
    for (int32_t t = 0; t < L - 1; ++t)
        for (int32_t s = 0; s < L - 1; ++s) {
            int64_t o = (int64_t)t * (L - 1) + s;
            double P1 = 0.0, P2 = 0.0;
            int64_t c1 = 0, c2 = 0;
            for (int32_t i = 0; i <= t; ++i)
                for (int32_t j = 0; j <= s; ++j) { P1 += (double)h[i * L + j] / (double)N; c1 += h[i * L + j]; }
            for (int32_t i = t + 1; i < L; ++i)
                for (int32_t j = s + 1; j < L; ++j) { P2 += (double)h[i * L + j] / (double)N; c2 += h[i * L + j]; }
            if (c1 == 0 || c2 == 0) { phi[o] = 0.0; valid[o] = 0; continue; }
            double H1 = 0.0, H2 = 0.0, s1 = 0.0, s2 = 0.0;
            for (int32_t i = 0; i <= t; ++i)
                for (int32_t j = 0; j <= s; ++j) {
                    double r = ((double)h[i * L + j] / (double)N) / P1;
                    if (alpha == 1.0) { if (r > 0) H1 -= r * log(r); } else s1 += pow(r, alpha);
                }
            for (int32_t i = t + 1; i < L; ++i)
                for (int32_t j = s + 1; j < L; ++j) {
                    double r = ((double)h[i * L + j] / (double)N) / P2;
                    if (alpha == 1.0) { if (r > 0) H2 -= r * log(r); } else s2 += pow(r, alpha);
                }
            if (alpha != 1.0) { H1 = tsallis_from_sum(s1, alpha); H2 = tsallis_from_sum(s2, alpha); }
            phi[o] = pseudo_additive(H1, H2, alpha);
            valid[o] = 1;
        }
    return 0;
}

/*
 * Plain-prefix mode of the 2-D form: two-dimensional running sums of p and
 * p^alpha from the (0,0) corner for quadrant 1 and from the (L-1,L-1) corner
 * for quadrant 2 (no subtraction from totals). O(L^2).
 */
int oracle_objective2d_prefix(const int64_t* h, int32_t L, double alpha, double* phi, uint8_t* valid) {
    if (!h || !phi || !valid || L < 2 || !(alpha > 0.0) || !isfinite(alpha)) return 1;
    int64_t LL = (int64_t)L * L;
    int64_t N = 0;
    for (int64_t k = 0; k < LL; ++k) N += h[k];
    double* A = (double*)calloc((size_t)LL * 4, sizeof(double));
    int64_t* C = (int64_t*)calloc((size_t)LL * 2, sizeof(int64_t));
    if (!A || !C) { free(A); free(C); return 2; }
    double *PA = A, *SA = A + LL, *PB = A + 2 * LL, *SB = A + 3 * LL;
    int64_t *CA = C, *CB = C + LL;
    /* quadrant-1 sums: X[i][j] = sum_{i'<=i, j'<=j} */
    for (int32_t i = 0; i < L; ++i) {
        double rp = 0.0, rs = 0.0;
        int64_t rc = 0;
        for (int32_t j = 0; j < L; ++j) {
            double p = N > 0 ? (double)h[i * L + j] / (double)N : 0.0;
            rp += p;
            rc += h[i * L + j];
            if (p > 0) rs += alpha == 1.0 ? p * log(p) : pow(p, alpha);
            int64_t o = (int64_t)i * L + j;
            PA[o] = rp + (i > 0 ? PA[o - L] : 0.0);
            SA[o] = rs + (i > 0 ? SA[o - L] : 0.0);
            CA[o] = rc + (i > 0 ? CA[o - L] : 0);
        }
    }
    /* quadrant-2 sums: Y[i][j] = sum_{i'>=i, j'>=j} */
    for (int32_t i = L - 1; i >= 0; --i) {
        double rp = 0.0, rs = 0.0;
        int64_t rc = 0;
        for (int32_t j = L - 1; j >= 0; --j) {
            double p = N > 0 ? (double)h[i * L + j] / (double)N : 0.0;
            rp += p;
            rc += h[i * L + j];
            if (p > 0) rs += alpha == 1.0 ? p * log(p) : pow(p, alpha);
            int64_t o = (int64_t)i * L + j;
            PB[o] = rp + (i < L - 1 ? PB[o + L] : 0.0);
            SB[o] = rs + (i < L - 1 ? SB[o + L] : 0.0);
            CB[o] = rc + (i < L - 1 ? CB[o + L] : 0);
        }
    }
    for (int32_t t = 0; t < L - 1; ++t)
        for (int32_t s = 0; s < L - 1; ++s) {
            int64_t o = (int64_t)t * (L - 1) + s;
            int64_t a = (int64_t)t * L + s, b = (int64_t)(t + 1) * L + (s + 1);
            if (CA[a] == 0 || CB[b] == 0) { phi[o] = 0.0; valid[o] = 0; continue; }
            double H1, H2;
            if (alpha == 1.0) {
                H1 = log(PA[a]) - SA[a] / PA[a];
                H2 = log(PB[b]) - SB[b] / PB[b];
            } else {
                H1 = tsallis_from_sum(SA[a] / pow(PA[a], alpha), alpha);
                H2 = tsallis_from_sum(SB[b] / pow(PB[b], alpha), alpha);
            }
            phi[o] = pseudo_additive(H1, H2, alpha);
            valid[o] = 1;
        }
    free(A);
    free(C);
    return 0;
}

/* ------------------------------------------------------------ argmax */

/*
 * The maximiser of phi_alpha (section II-C, last equation): the smallest t
 * attaining the maximum over valid thresholds. Also reports the relative gap
 * to the best value among thresholds that give a different partition
 * (a different class-1 count), or +inf when there is none. Returns t = -1
 * when no threshold is valid.
 */
int oracle_argmax1d(const double* phi, const uint8_t* valid, const int64_t* h, int32_t L,
                    int32_t* t_out, double* best_out, double* gap_out) {
    if (!phi || !valid || !h || !t_out || L < 2) return 1;
    int32_t bt = -1;
    double best = 0.0;
    for (int32_t t = 0; t < L - 1; ++t)
        if (valid[t] && (bt < 0 || phi[t] > best)) { best = phi[t]; bt = t; }
    *t_out = bt;
    if (best_out) *best_out = bt >= 0 ? best : 0.0;
    if (gap_out) {
        double second = -INFINITY;
        int64_t nbest = 0, n = 0;
        for (int32_t i = 0; i <= bt && bt >= 0; ++i) nbest += h[i];
        for (int32_t t = 0; t < L - 1; ++t) {
            n += h[t];
            if (valid[t] && n != nbest && phi[t] > second) second = phi[t];
        }
        double scale = fabs(best) > 1.0 ? fabs(best) : 1.0;
        *gap_out = (bt < 0 || second == -INFINITY) ? INFINITY : (best - second) / scale;
    }
    return 0;
}

/* 2-D maximiser: smallest t, then smallest s. Partitions are told apart by
 * their (class-1 count, class-2 count) pair. */
int oracle_argmax2d(const double* phi, const uint8_t* valid, const int64_t* h, int32_t L,
                    int32_t* t_out, int32_t* s_out, double* best_out, double* gap_out) {
    if (!phi || !valid || !h || !t_out || !s_out || L < 2) return 1;
    int32_t bt = -1, bs = -1;
    double best = 0.0;
    for (int32_t t = 0; t < L - 1; ++t)
        for (int32_t s = 0; s < L - 1; ++s) {
            int64_t o = (int64_t)t * (L - 1) + s;
            if (valid[o] && (bt < 0 || phi[o] > best)) { best = phi[o]; bt = t; bs = s; }
        }
    *t_out = bt;
    *s_out = bs;
    if (best_out) *best_out = bt >= 0 ? best : 0.0;
    if (gap_out) {
        if (bt < 0) { *gap_out = INFINITY; return 0; }
        int64_t LL = (int64_t)L * L;
        int64_t* CA = (int64_t*)calloc((size_t)LL * 2, sizeof(int64_t));
        if (!CA) return 2;
        int64_t* CB = CA + LL;
        for (int32_t i = 0; i < L; ++i)
            for (int32_t j = 0; j < L; ++j) {
                int64_t o = (int64_t)i * L + j;
                CA[o] = h[o] + (i > 0 ? CA[o - L] : 0) + (j > 0 ? CA[o - 1] : 0) - (i > 0 && j > 0 ? CA[o - L - 1] : 0);
            }
        for (int32_t i = L - 1; i >= 0; --i)
            for (int32_t j = L - 1; j >= 0; --j) {
                int64_t o = (int64_t)i * L + j;
                CB[o] = h[o] + (i < L - 1 ? CB[o + L] : 0) + (j < L - 1 ? CB[o + 1] : 0) -
                        (i < L - 1 && j < L - 1 ? CB[o + L + 1] : 0);
            }
        int64_t ka = CA[(int64_t)bt * L + bs], kb = CB[(int64_t)(bt + 1) * L + bs + 1];
        double second = -INFINITY;
        for (int32_t t = 0; t < L - 1; ++t)
            for (int32_t s = 0; s < L - 1; ++s) {
                int64_t o = (int64_t)t * (L - 1) + s;
                if (!valid[o]) continue;
                if (CA[(int64_t)t * L + s] == ka && CB[(int64_t)(t + 1) * L + s + 1] == kb) continue;
                if (phi[o] > second) second = phi[o];
            }
        double scale = fabs(best) > 1.0 ? fabs(best) : 1.0;
        *gap_out = second == -INFINITY ? INFINITY : (best - second) / scale;
        free(CA);
    }
    return 0;
}

/* ------------------------------------------------------------ binarise */

/* Algorithm 1, thresholding kernel: a voxel is foreground when its level is
 * >= T. polarity 1 is that literal form with T = t + 1 (class 2 is
 * foreground); polarity 0 marks class 1 (levels <= t), the low-HU airway
 * lumen. Levels are the 1-D bins b = clamp(v - lo, 0, L-1), or the 2-D grey
 * levels b >> shift when shift > 0. */
int oracle_binarize(const int16_t* vol, int64_t n, int32_t lo, int32_t L, int32_t shift, int32_t t,
                    int32_t polarity, uint8_t* mask) {
    if (!vol || !mask || n < 0) return 1;
    for (int64_t k = 0; k < n; ++k) {
        int32_t b = (int32_t)vol[k] - lo;
        if (b < 0) b = 0;
        if (b > L - 1) b = L - 1;
        b >>= shift;
        int fg = polarity ? (b >= t + 1) : (b <= t);
        mask[k] = (uint8_t)(t >= 0 ? fg : 0);
    }
    return 0;
}

/* ------------------------------------------------------------ whole step */

typedef struct {
    const int16_t* vol;
    int64_t nvox_group;
    int32_t lo, L, polarity, definition;
    double alpha;
    int64_t g0, g1;
    int32_t* t_out;
    double* phi_out;
    double* gap_out;
    uint8_t* mask;
    int rc;
} seg_job;

static void* seg_worker(void* arg) {
    seg_job* j = (seg_job*)arg;
    int64_t* h = (int64_t*)malloc(sizeof(int64_t) * (size_t)j->L);
    double* phi = (double*)malloc(sizeof(double) * (size_t)j->L);
    uint8_t* valid = (uint8_t*)malloc((size_t)j->L);
    if (!h || !phi || !valid) { j->rc = 2; free(h); free(phi); free(valid); return NULL; }
    for (int64_t g = j->g0; g < j->g1 && j->rc == 0; ++g) {
        const int16_t* v = j->vol + g * j->nvox_group;
        int rc = oracle_hist1d(v, j->nvox_group, j->lo, j->L, h);
        if (!rc) rc = j->definition ? oracle_objective1d_def(h, j->L, j->alpha, phi, valid)
                                    : oracle_objective1d_prefix(h, j->L, j->alpha, phi, valid);
        int32_t t = -1;
        double best = 0.0, gap = 0.0;
        if (!rc) rc = oracle_argmax1d(phi, valid, h, j->L, &t, &best, &gap);
        if (!rc && j->mask) rc = oracle_binarize(v, j->nvox_group, j->lo, j->L, 0, t, j->polarity,
                                                 j->mask + g * j->nvox_group);
        j->t_out[g] = t;
        if (j->phi_out) j->phi_out[g] = best;
        if (j->gap_out) j->gap_out[g] = gap;
        j->rc = rc;
    }
    free(h); free(phi); free(valid);
    return NULL;
}

/*
 * The whole 1-D step (histogram, objective, maximiser, Algorithm 1) for
 * ngroups consecutive groups of nvox_group voxels each (a slice, a volume),
 * spread over nthreads host threads, one group at a time per thread.
 */
int oracle_segment1d(const int16_t* vol, int64_t nvox_group, int64_t ngroups, int32_t lo, int32_t L,
                     double alpha, int32_t polarity, int32_t definition, int32_t nthreads,
                     int32_t* t_out, double* phi_out, double* gap_out, uint8_t* mask) {
    if (!vol || !t_out || nvox_group < 1 || ngroups < 1 || L < 2) return 1;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > ngroups) nthreads = (int32_t)ngroups;
    seg_job* jobs = (seg_job*)calloc((size_t)nthreads, sizeof(seg_job));
    pthread_t* th = (pthread_t*)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!jobs || !th) { free(jobs); free(th); return 2; }
    for (int32_t i = 0; i < nthreads; ++i) {
        seg_job* j = &jobs[i];
        j->vol = vol; j->nvox_group = nvox_group; j->lo = lo; j->L = L; j->polarity = polarity;
        j->definition = definition; j->alpha = alpha;
        j->g0 = ngroups * i / nthreads; j->g1 = ngroups * (i + 1) / nthreads;
        j->t_out = t_out; j->phi_out = phi_out; j->gap_out = gap_out; j->mask = mask; j->rc = 0;
    }
    int32_t started = 0;
    int rc = 0;
    for (int32_t i = 1; i < nthreads; ++i) {
        if (pthread_create(&th[i], NULL, seg_worker, &jobs[i]) != 0) { rc = 3; break; }
        started = i;
    }
    if (rc == 0) seg_worker(&jobs[0]);
    for (int32_t i = 1; i <= started; ++i) pthread_join(th[i], NULL);
    for (int32_t i = 0; i < nthreads && rc == 0; ++i) rc = jobs[i].rc;
    free(jobs);
    free(th);
    return rc;
}

/* ------------------------------------------------------------ pre-processing */

/*
 * Section II-B "Pre-processing": the CT numbers are turned into an 8-bit
 * grey image. Readings (the text gives no formula): a voxel at or below the
 * detector background value (-2000 HU) becomes 0; every other value is
 * clamped to [hu_min, hu_max] (by default the histogram range of Fig. 3,
 * -2000..2500) and mapped linearly onto 0..255, rounded to the nearest level
 * with halves rounded up: g = floor((v - hu_min) * 255 / (hu_max - hu_min) + 1/2),
 * computed here in exact integer arithmetic.
 */
int oracle_rescale8(const int16_t* vol, int64_t n, int32_t background, int32_t hu_min, int32_t hu_max,
                    uint8_t* out) {
    if (!vol || !out || n < 0 || hu_max <= hu_min) return 1;
    const int64_t D = (int64_t)hu_max - hu_min;
    for (int64_t k = 0; k < n; ++k) {
        int64_t v = vol[k];
        if (v <= background) { out[k] = 0; continue; }
        if (v < hu_min) v = hu_min;
        if (v > hu_max) v = hu_max;
        /* (v - hu_min) * 255 / D + 1/2, floored: numerator and denominator doubled */
        int64_t g = (2 * (v - hu_min) * 255 + D) / (2 * D);
        out[k] = (uint8_t)g;
    }
    return 0;
}

/*
 * Section II-C "Morphology": erosion and dilation of the grey image A by a
 * flat structuring element B, opening (erosion, then dilation), and the
 * chest-mask subtraction. B is the digital disk of radius r: the offsets
 * (dx, dy) with dx^2 + dy^2 <= r^2 (r = 10 reads the paper's disk of size 10
 * pixels). Flat grey erosion is the minimum of A over B placed at the pixel,
 * dilation the maximum (B is symmetric, so B and its reflection agree).
 * Offsets that leave the image are not part of the window. Each slice (z) is
 * a separate 2-D image, as in the paper.
 *
 * op: 1 erosion, 2 dilation, 3 opening, 4 closing (dilation, then erosion),
 * 5 chest-mask subtraction A - opening(A), 6 closing(A) - A. The text
 * subtracts the image from its opening; an opening never exceeds the image,
 * so that difference is read with the sign that leaves it non-negative
 * (op 5). op 0 copies A.
 */
static void morph_pass(const uint8_t* in, int64_t nx, int64_t ny, int32_t r, int use_max, uint8_t* out) {
    for (int64_t y = 0; y < ny; ++y)
        for (int64_t x = 0; x < nx; ++x) {
            int v = use_max ? 0 : 255;
            for (int32_t dy = -r; dy <= r; ++dy)
                for (int32_t dx = -r; dx <= r; ++dx) {
                    if (dx * dx + dy * dy > r * r) continue;
                    int64_t xx = x + dx, yy = y + dy;
                    if (xx < 0 || xx >= nx || yy < 0 || yy >= ny) continue;
                    int a = in[yy * nx + xx];
                    if (use_max ? a > v : a < v) v = a;
                }
            out[y * nx + x] = (uint8_t)v;
        }
}

int oracle_morph2d(const uint8_t* img, int64_t nx, int64_t ny, int64_t nz, int32_t r, int32_t op, uint8_t* out) {
    if (!img || !out || nx < 1 || ny < 1 || nz < 0 || r < 0 || op < 0 || op > 6) return 1;
    const int64_t ns = nx * ny;
    uint8_t* a = (uint8_t*)malloc((size_t)ns);
    uint8_t* b = (uint8_t*)malloc((size_t)ns);
    if (!a || !b) { free(a); free(b); return 2; }
    for (int64_t z = 0; z < nz; ++z) {
        const uint8_t* A = img + z * ns;
        uint8_t* O = out + z * ns;
        switch (op) {
            case 0: memcpy(O, A, (size_t)ns); break;
            case 1: morph_pass(A, nx, ny, r, 0, O); break;
            case 2: morph_pass(A, nx, ny, r, 1, O); break;
            case 3: morph_pass(A, nx, ny, r, 0, a); morph_pass(a, nx, ny, r, 1, O); break;
            case 4: morph_pass(A, nx, ny, r, 1, a); morph_pass(a, nx, ny, r, 0, O); break;
            case 5:
                morph_pass(A, nx, ny, r, 0, a); morph_pass(a, nx, ny, r, 1, b);
                for (int64_t k = 0; k < ns; ++k) O[k] = (uint8_t)(A[k] - b[k]);
                break;
            case 6:
                morph_pass(A, nx, ny, r, 1, a); morph_pass(a, nx, ny, r, 0, b);
                for (int64_t k = 0; k < ns; ++k) O[k] = (uint8_t)(b[k] - A[k]);
                break;
        }
    }
    free(a); free(b);
    return 0;
}
