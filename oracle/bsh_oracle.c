/*
 * bsh_oracle.c -- plain FP64 CPU oracle for the BinarySkyHough number count.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the package smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant generator with the CUDA path.
 *
 * Everything is computed directly from the definitions in the paper
 * (Covas & Sintes, "BinarySkyHough", arXiv:1904.04873), template by
 * template, in double precision, with no tiling and no look-up tables:
 *
 *   peakgram      Eq. (20)-(21) and the 1/0 threshold of Sec. IV.A
 *   weights       Eq. (22), antenna patterns of Eq. (1)
 *   track         Eq. (15) multiplied by T_c, rounded to the nearest bin;
 *                 Eq. (14) (ELL1, first order in e) for eccentric grids
 *   number count  Sec. IV.C: weighted sum of 1s and 0s along the track
 *   significance  Eq. (25)
 *   toplist       Sec. IV.C: per-region list ranked by s_H
 *   power sum     Eq. (26): weighted sum of rho along the exact track
 *
 * Build with -O2 -ffp-contract=off so that no multiply-add is fused.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_ARG 1
#define ORC_ERR_RANGE 2

/* ------------------------------------------------------------------------ */
/* Peakgram: Eq. (20) rho = |x|^2 / <n>^2, with <n>^2 estimated by a running  */
/* median over `window` bins (Sec. IV.A).  For Exp(1) powers the median is   */
/* ln 2, so <n>^2 = median / ln 2.  Bins with rho > rho_th become 1.         */
/* ------------------------------------------------------------------------ */

static int cmp_float(const void* a, const void* b) {
    float x = *(const float*)a, y = *(const float*)b;
    return (x < y) ? -1 : (x > y) ? 1 : 0;
}

/* Median of the window centred on bin k; near the edges the window is
 * shifted (not truncated) to stay inside [0, K). */
double orc_running_median(const float* row, int K, int window, int k) {
    int half = window / 2;
    int a = k - half;
    if (a < 0) a = 0;
    if (a + window > K) a = K - window;
    float* buf = (float*)malloc(sizeof(float) * (size_t)window);
    memcpy(buf, row + a, sizeof(float) * (size_t)window);
    qsort(buf, (size_t)window, sizeof(float), cmp_float);
    double m = (double)buf[window / 2];
    free(buf);
    return m;
}

int orc_peakgram(const float* power, int N, int K, int window, double rho_th,
                 float* rho_out, uint32_t* bits, int W) {
    if (N < 0 || K <= 0 || W * 32 < K) return ORC_ERR_ARG;
    if (window != 0 && (window % 2 == 0 || window > K)) return ORC_ERR_ARG;
    const double ln2 = 0.69314718055994530942;
    memset(bits, 0, sizeof(uint32_t) * (size_t)N * (size_t)W);
    for (int i = 0; i < N; ++i) {
        const float* row = power + (size_t)i * K;
        for (int k = 0; k < K; ++k) {
            double P = (double)row[k];
            int on;
            double rho;
            if (window == 0) {
                rho = P;
                on = P > rho_th;
            } else {
                double m = orc_running_median(row, K, window, k);
                /* rho > rho_th  <=>  P ln2 > rho_th m  (m > 0) */
                double lhs = P * ln2;
                double rhs = rho_th * m;
                on = lhs > rhs;
                rho = lhs / m;
            }
            if (rho_out) rho_out[(size_t)i * K + k] = (float)rho;
            if (on) bits[(size_t)i * W + (k >> 5)] |= (uint32_t)1u << (k & 31);
        }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Antenna patterns F+, Fx (Eq. (1), from the Jaranowski-Krolak-Schutz      */
/* formalism cited there).  Detector tensor D = (u u^T - v v^T)/2 for arm   */
/* unit vectors u, v; polarisation tensors e+ = p p^T - q q^T and           */
/* ex = p q^T + q p^T for an orthonormal pair (p, q) orthogonal to the      */
/* propagation direction, rotated by the polarisation angle psi.            */
/* ------------------------------------------------------------------------ */

static double dot3(const double* a, const double* b) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

void orc_antenna(const double* n, const double* u, const double* v, double psi,
                 double* Fp, double* Fc) {
    /* basis orthogonal to n: e_alpha = z x n / |z x n|, e_delta = n x e_alpha */
    double nx = n[0], ny = n[1], nz = n[2];
    double rxy = sqrt(nx * nx + ny * ny);
    double ea[3], ed[3];
    if (rxy > 1e-300) {
        ea[0] = -ny / rxy; ea[1] = nx / rxy; ea[2] = 0.0;
    } else {
        ea[0] = 0.0; ea[1] = 1.0; ea[2] = 0.0;
    }
    ed[0] = ny * ea[2] - nz * ea[1];
    ed[1] = nz * ea[0] - nx * ea[2];
    ed[2] = nx * ea[1] - ny * ea[0];
    double c = cos(psi), s = sin(psi);
    double p[3], q[3];
    for (int k = 0; k < 3; ++k) {
        p[k] = c * ea[k] + s * ed[k];
        q[k] = -s * ea[k] + c * ed[k];
    }
    double up = dot3(u, p), uq = dot3(u, q), vp = dot3(v, p), vq = dot3(v, q);
    /* D : e+ and D : ex with D = (u u - v v)/2 */
    *Fp = 0.5 * ((up * up - uq * uq) - (vp * vp - vq * vq));
    *Fc = up * uq - vp * vq;
}

/* Weights, Eq. (22): w_J proportional to (F+^2 + Fx^2)/S_n at the SFT mid-time.
 * arms: [N][6] (u then v) at each SFT mid-time; Sn: [N].  norm = 1 scales the
 * weights of each sky point so that they sum to N. */
int orc_weights(const double* sky, int S, const double* arms, const double* Sn, int N,
                int norm, double* w) {
    if (S < 0 || N <= 0) return ORC_ERR_ARG;
    for (int s = 0; s < S; ++s) {
        double sum = 0.0;
        for (int i = 0; i < N; ++i) {
            double Fp, Fc;
            orc_antenna(sky + 3 * (size_t)s, arms + 6 * (size_t)i, arms + 6 * (size_t)i + 3, 0.0, &Fp, &Fc);
            double x = (Fp * Fp + Fc * Fc) / Sn[i];
            w[(size_t)s * N + i] = x;
            sum += x;
        }
        if (norm) {
            if (!(sum > 0.0)) return ORC_ERR_RANGE;
            for (int i = 0; i < N; ++i) w[(size_t)s * N + i] = w[(size_t)s * N + i] * ((double)N / sum);
        }
    }
    return ORC_OK;
}

/* Round a double to the nearest value of a binary floating-point format
 * with `mant` explicit mantissa bits, minimum normal exponent `emin` and
 * maximum finite value `maxv`, ties to even (IEEE 754 roundTiesToEven).
 * half: (10, -14, 65504); bfloat16: (7, -126, 3.3895313892515355e38);
 * single: (23, -126, 3.4028234663852886e38). */
static double round_format(double x, int mant, int emin, double maxv) {
    if (x == 0.0 || isnan(x) || isinf(x)) return x;
    double ax = fabs(x);
    int e;
    frexp(ax, &e);          /* ax = f * 2^e, f in [0.5, 1) */
    int E = e - 1;          /* ax in [2^E, 2^(E+1)) */
    if (E < emin) E = emin; /* subnormal range: fixed quantum */
    double quantum = ldexp(1.0, E - mant);
    double q = ax / quantum;              /* exact: power-of-two scaling */
    double r = floor(q);
    double frac = q - r;
    if (frac > 0.5 || (frac == 0.5 && fmod(r, 2.0) != 0.0)) r += 1.0;
    double y = r * quantum;
    if (y > maxv) y = INFINITY;
    return x < 0 ? -y : y;
}

double orc_round_f16(double x) { return round_format(x, 10, -14, 65504.0); }
double orc_round_bf16(double x) { return round_format(x, 7, -126, 3.3895313892515355e38); }
double orc_round_f32(double x) { return round_format(x, 23, -126, 3.4028234663852886e38); }

/* dtype: 0 = f64, 1 = f32, 2 = f16, 3 = bf16 */
void orc_quantize(const double* in, double* out, size_t n, int dtype) {
    for (size_t k = 0; k < n; ++k) {
        double x = in[k];
        switch (dtype) {
            case 1: x = orc_round_f32(x); break;
            case 2: x = orc_round_f16(x); break;
            case 3: x = orc_round_bf16(x); break;
            default: break;
        }
        out[k] = x;
    }
}

/* ------------------------------------------------------------------------ */
/* Track, Eq. (15) times T_c:                                               */
/*   f(t)T = F (1 + v.n - a_p Omega cos(Omega (t - t_asc))),  F = f0 T        */
/* evaluated in this order (double precision, no fused multiply-add):       */
/*   vn = (v.x n.x + v.y n.y) + v.z n.z                                      */
/*   c  = cos(Omega (t - t_asc));  D = vn - a_p (Omega c)                    */
/*   x  = F + F D;                 k = floor(x + 1/2)                        */
/* `tie` is set when x lies within tie_band of a half-integer, where the    */
/* rounding could go either way between two correct FP64 evaluations.       */
/* ------------------------------------------------------------------------ */

double orc_track_x(double F, const double* v, const double* n, double ap, double Om,
                   double Tasc, double t) {
    double vn = (v[0] * n[0] + v[1] * n[1]) + v[2] * n[2];
    double c = cos(Om * (t - Tasc));
    double D = vn - ap * (Om * c);
    return F + F * D;
}

int64_t orc_track_bin(double F, const double* v, const double* n, double ap, double Om,
                      double Tasc, double t, double tie_band, int* tie) {
    double x = orc_track_x(F, v, n, ap, Om, Tasc, t);
    double fr = x - floor(x);
    if (tie) *tie = fabs(fr - 0.5) < tie_band;
    return (int64_t)floor(x + 0.5);
}

/* Low-eccentricity (ELL1) track, first order in e (Eq. (14), Sec. II):       */
/*   f(t)T = F (1 + v.n - a_p Omega g),                                      */
/*   g = cos(phi) + kappa cos(2 phi) + eta sin(2 phi),  phi = Omega (t - t_asc)  */
/* with kappa = e cos(omega), eta = e sin(omega).  The sign of the eta term   */
/* is the one the paper's exact Keplerian orbit (Eq. (6)-(10)) gives at       */
/* first order in e; Eq. (14) as printed carries the opposite sign.  With    */
/* kappa = eta = 0, g = cos(phi) exactly and the circular track is recovered */
/* bit for bit.  Evaluation order: vn as above, phi = Omega (t - t_asc),     */
/* g = (cos(phi) + kappa cos(2 phi)) + eta sin(2 phi), D = vn - a_p (Omega g). */
double orc_track_x_ell1(double F, const double* v, const double* n, double ap, double Om,
                        double Tasc, double kap, double eta, double t) {
    double vn = (v[0] * n[0] + v[1] * n[1]) + v[2] * n[2];
    double phi = Om * (t - Tasc);
    double g = (cos(phi) + kap * cos(2.0 * phi)) + eta * sin(2.0 * phi);
    double D = vn - ap * (Om * g);
    return F + F * D;
}

int64_t orc_track_bin_ell1(double F, const double* v, const double* n, double ap, double Om,
                           double Tasc, double kap, double eta, double t, double tie_band, int* tie) {
    double x = orc_track_x_ell1(F, v, n, ap, Om, Tasc, kap, eta, t);
    double fr = x - floor(x);
    if (tie) *tie = fabs(fr - 0.5) < tie_band;
    return (int64_t)floor(x + 0.5);
}

/* ------------------------------------------------------------------------ */
/* One band searched over a sky set and a binary grid.                      */
/* Template order: id = ((s * B + b) * n_f0 + j), F_j = F0 + j,            */
/* b = (((iOm * n_T + iT) * n_kap + ik) * n_eta + ie) * n_ap + iap.          */
/* n_kap = n_eta = 0 means one value 0 each (circular orbits).              */
/* ------------------------------------------------------------------------ */

typedef struct {
    int N;                 /* SFTs */
    int k_lo, K, W;        /* loaded band and words per bit row */
    const uint32_t* bits;  /* [N][W] */
    const float* rho;      /* [N][K] or NULL */
    const double* w;       /* [S][N] weights (already quantised if desired) */
    const double* v;       /* [N][3] */
    const double* t;       /* [N] */
    double F0;
    int n_f0;
    int S;
    const double* sky;     /* [S][3] */
    int n_ap;
    const double* ap;
    int n_Om;
    const double* Om;
    int n_T;
    const double* Tasc;    /* [n_Om][n_T] */
    double rho_th;
    double tie_band;
    int n_kap;
    const double* kap;    /* [n_kap] e cos(omega), or NULL with n_kap = 0 */
    int n_eta;
    const double* eta;    /* [n_eta] e sin(omega), or NULL with n_eta = 0 */
    int lut_block;        /* 0: exact track; L > 0: look-up-table approximation, blocks of L f0 */
    /* explicit binary bank: n_orbit > 0 selects it and the grid above is ignored;
       binary template b has a_p = bank_ap[b] and the orbit row bank_orbit[b] */
    int n_orbit;
    const double* orbit;      /* [n_orbit][4]: Omega, t_asc, kappa, eta */
    int64_t n_bank;
    const int32_t* bank_orbit;/* [n_bank] */
    const double* bank_ap;    /* [n_bank] */
} orc_problem;

/* Look-up-table approximation of stage 1 (Sec. IV.B): the modulation F D of  */
/* the track is evaluated once per block of L contiguous f0 templates, at the */
/* block's reference template, and reused for the other templates of the      */
/* block, whose bins are the reference bins shifted by their f0 offset:       */
/*   k_j = floor(F_ref + F_ref D + 1/2) + (j - j_ref).                        */
/* Block q holds j in [qL, min(qL + L, n_f0)); its reference is its middle    */
/* template j_ref = qL + (len - 1)/2 (len = the block's length, integer       */
/* division).  L = 1 is the exact track.                                      */
static int lut_ref(const orc_problem* pr, int j) {
    int L = pr->lut_block;
    int q = j / L;
    int len = pr->n_f0 - q * L;
    if (len > L) len = L;
    return q * L + (len - 1) / 2;
}

static void template_params(const orc_problem* pr, int64_t b, double* ap, double* Om, double* Ta,
                            double* kap, double* eta) {
    if (pr->n_orbit > 0) {
        const double* o = pr->orbit + 4 * (size_t)pr->bank_orbit[b];
        *ap = pr->bank_ap[b];
        *Om = o[0];
        *Ta = o[1];
        *kap = o[2];
        *eta = o[3];
        return;
    }
    int nk = pr->n_kap > 0 ? pr->n_kap : 1;
    int ne = pr->n_eta > 0 ? pr->n_eta : 1;
    int64_t iap = b % pr->n_ap;
    int64_t r = b / pr->n_ap;
    int64_t ie = r % ne;
    r /= ne;
    int64_t ik = r % nk;
    r /= nk;
    int64_t iT = r % pr->n_T;
    int64_t iOm = r / pr->n_T;
    *ap = pr->ap[iap];
    *Om = pr->Om[iOm];
    *Ta = pr->Tasc[iOm * pr->n_T + iT];
    *kap = pr->n_kap > 0 ? pr->kap[ik] : 0.0;
    *eta = pr->n_eta > 0 ? pr->eta[ie] : 0.0;
}

/* Number count of one template (Sec. IV.C): n = sum_i w_i * bit_i[k_i].
 * Returns ORC_ERR_RANGE when a track leaves the loaded band.  Also returns
 * the smallest / largest counts reachable by rounding each tie-flagged term
 * to either neighbouring bin. */
int orc_count_one(const orc_problem* pr, int s, int64_t b, int j,
                  int32_t* n_unw, double* n_w, int32_t* n_tie,
                  int32_t* unw_lo, int32_t* unw_hi, double* w_lo, double* w_hi) {
    double ap, Om, Ta, kap, eta;
    template_params(pr, b, &ap, &Om, &Ta, &kap, &eta);
    /* the track is evaluated at F (exact) or at the block's reference F_ref (LUT) */
    int shift = 0;
    if (pr->lut_block > 0) {
        int jr = lut_ref(pr, j);
        shift = j - jr;
        j = jr;
    }
    double F = pr->F0 + (double)j;
    const double* n = pr->sky + 3 * (size_t)s;
    int32_t cu = 0, ties = 0, lo = 0, hi = 0;
    double cw = 0.0, wl = 0.0, wh = 0.0;
    for (int i = 0; i < pr->N; ++i) {
        int tie;
        int64_t k = orc_track_bin_ell1(F, pr->v + 3 * (size_t)i, n, ap, Om, Ta, kap, eta, pr->t[i],
                                       pr->tie_band, &tie) + shift;
        int64_t col = k - pr->k_lo;
        if (col < 0 || col >= pr->K) return ORC_ERR_RANGE;
        const uint32_t* row = pr->bits + (size_t)i * pr->W;
        int bit = (int)((row[col >> 5] >> (col & 31)) & 1u);
        double wi = pr->w[(size_t)s * pr->N + i];
        cu += bit;
        if (bit) cw += wi;
        if (tie) {
            /* the other candidate bin: the neighbour on the far side of the half */
            double x = orc_track_x_ell1(F, pr->v + 3 * (size_t)i, n, ap, Om, Ta, kap, eta, pr->t[i]);
            int64_t alt = (x + 0.5 - floor(x + 0.5) < 0.5) ? k - 1 : k + 1;
            int64_t ca = alt - pr->k_lo;
            int abit = 0;
            if (ca >= 0 && ca < pr->K) abit = (int)((row[ca >> 5] >> (ca & 31)) & 1u);
            ++ties;
            int mn = bit < abit ? bit : abit, mx = bit > abit ? bit : abit;
            lo += mn; hi += mx;
            wl += mn ? wi : 0.0; wh += mx ? wi : 0.0;
        } else {
            lo += bit; hi += bit;
            if (bit) { wl += wi; wh += wi; }
        }
    }
    if (n_unw) *n_unw = cu;
    if (n_w) *n_w = cw;
    if (n_tie) *n_tie = ties;
    if (unw_lo) *unw_lo = lo;
    if (unw_hi) *unw_hi = hi;
    if (w_lo) *w_lo = wl;
    if (w_hi) *w_hi = wh;
    return ORC_OK;
}

/* All templates of sky points [s_begin, s_end), in template order. */
int orc_count_dense(const orc_problem* pr, int s_begin, int s_end,
                    int32_t* n_unw, double* n_w, int32_t* n_tie,
                    int32_t* unw_lo, int32_t* unw_hi, double* w_lo, double* w_hi) {
    int64_t B = pr->n_orbit > 0 ? pr->n_bank
                                : (int64_t)pr->n_ap * pr->n_Om * pr->n_T * (pr->n_kap > 0 ? pr->n_kap : 1) *
                                      (pr->n_eta > 0 ? pr->n_eta : 1);
    size_t idx = 0;
    for (int s = s_begin; s < s_end; ++s)
        for (int64_t b = 0; b < B; ++b)
            for (int j = 0; j < pr->n_f0; ++j, ++idx) {
                int rc = orc_count_one(pr, s, b, j, n_unw ? n_unw + idx : 0, n_w ? n_w + idx : 0,
                                       n_tie ? n_tie + idx : 0, unw_lo ? unw_lo + idx : 0,
                                       unw_hi ? unw_hi + idx : 0, w_lo ? w_lo + idx : 0,
                                       w_hi ? w_hi + idx : 0);
                if (rc) return rc;
            }
    return ORC_OK;
}

/* Eq. (25): s_H = (n - <n>)/sigma with, for independent weighted Bernoulli(p)
 * terms, <n> = p sum w and sigma^2 = p (1-p) sum w^2, p = exp(-rho_th). */
double orc_significance(double n, double sum_w, double sum_w2, double rho_th) {
    double p = exp(-rho_th);
    double mean = p * sum_w;
    double var = p * (1.0 - p) * sum_w2;
    if (!(var > 0.0)) return 0.0;
    return (n - mean) / sqrt(var);
}

/* ------------------------------------------------------------------------ */
/* Toplist (Sec. IV.C): per sky patch, the k templates with the largest s_H; */
/* equal scores are ordered by the smaller template id inside the patch.    */
/* ------------------------------------------------------------------------ */

typedef struct { double score; int64_t id; } orc_entry;

static int cmp_entry(const void* a, const void* b) {
    const orc_entry* x = (const orc_entry*)a;
    const orc_entry* y = (const orc_entry*)b;
    if (x->score > y->score) return -1;
    if (x->score < y->score) return 1;
    return (x->id < y->id) ? -1 : (x->id > y->id) ? 1 : 0;
}

/* scores: [n] in template order of one patch; out_ids/out_scores: [k].
 * Returns the number written (min(k, n)). */
int64_t orc_topk(const double* scores, int64_t n, int64_t k, int64_t* out_ids, double* out_scores) {
    orc_entry* e = (orc_entry*)malloc(sizeof(orc_entry) * (size_t)(n > 0 ? n : 1));
    for (int64_t q = 0; q < n; ++q) { e[q].score = scores[q]; e[q].id = q; }
    qsort(e, (size_t)n, sizeof(orc_entry), cmp_entry);
    int64_t m = n < k ? n : k;
    for (int64_t q = 0; q < m; ++q) { out_ids[q] = e[q].id; out_scores[q] = e[q].score; }
    free(e);
    return m;
}

/* ------------------------------------------------------------------------ */
/* Stage 2, Eq. (26): P = sum_i w_i rho_i[k_i] along the exact track,        */
/* s_P = (P - <P>)/sigma_P with <P> = sum w, sigma_P^2 = sum w^2 (rho of     */
/* Gaussian noise is Exp(1): mean 1, variance 1).                            */
/* ------------------------------------------------------------------------ */

int orc_power_sum(const orc_problem* pr, int s, int64_t b, int j, double* P) {
    double ap, Om, Ta, kap, eta;
    template_params(pr, b, &ap, &Om, &Ta, &kap, &eta);
    double F = pr->F0 + (double)j;
    const double* n = pr->sky + 3 * (size_t)s;
    double acc = 0.0;
    for (int i = 0; i < pr->N; ++i) {
        int64_t k = orc_track_bin_ell1(F, pr->v + 3 * (size_t)i, n, ap, Om, Ta, kap, eta, pr->t[i], 0.0, 0);
        int64_t col = k - pr->k_lo;
        if (col < 0 || col >= pr->K) return ORC_ERR_RANGE;
        acc += pr->w[(size_t)s * pr->N + i] * (double)pr->rho[(size_t)i * pr->K + col];
    }
    *P = acc;
    return ORC_OK;
}

double orc_power_significance(double P, double sum_w, double sum_w2) {
    if (!(sum_w2 > 0.0)) return 0.0;
    return (P - sum_w) / sqrt(sum_w2);
}
