/*
 * bsh.h -- C ABI of the GB300-native BinarySkyHough number count.
 *
 * Method: P. B. Covas and A. M. Sintes, "BinarySkyHough: a new method to
 * search for continuous gravitational waves from unknown neutron stars in
 * binary systems", arXiv:1904.04873.  Section / equation numbers below are
 * the paper's.
 *
 * Conventions for every entry point:
 *   - Array arguments are DEVICE pointers owned by the caller unless the
 *     comment says HOST.  The library never allocates device memory: the
 *     only device memory it uses besides the caller's arrays is the plan
 *     workspace the caller passes to bsh_plan_bind(), and the fixed-size
 *     static array behind bsh_power_sum_static().
 *   - Calls taking a stream only enqueue work on it (asynchronous).  Those
 *     marked "capturable" make no host synchronisation and no allocation and
 *     may be recorded into a CUDA graph.
 *   - Every call returns BSH_OK or one of the BSH_ERR_* codes below.
 *     Argument errors are detected on the host before anything is enqueued.
 *     Errors found by kernels (a track leaving the loaded band, a fixed-point
 *     table out of range, a bounded wait that expired) are recorded in a
 *     device status word and returned by bsh_sync_status().  No kernel traps
 *     or prints.
 *   - Row-major layouts: [a][b] means b is the fastest index.
 *   - Frequencies are bin numbers F = f * T_c (Eq. (33): delta f = 1/T_c).
 *   - Template order inside a problem: id = ((s * B + b) * n_f0 + j) with
 *     F_j = F0 + j and the binary index
 *       b = (((iOm * n_T + iT) * n_kap + ik) * n_eta + ie) * n_ap + iap
 *     for a grid, where n_kap (n_eta) counts as 1 when the problem gives no
 *     kappa (eta), or b = the entry of an explicit bank (bank_orbit, bank_ap).
 *   - Track of a template at SFT i (Eq. (14) and (15) times T_c):
 *       k_i = floor(F (1 + v_i.n - a_p Omega g_i) + 1/2),
 *       g_i = cos(phi) + kappa cos(2 phi) + eta sin(2 phi),
 *       phi = Omega (t_i - t_asc),  kappa = e cos(omega),  eta = e sin(omega),
 *     the low-eccentricity (ELL1) expansion to first order in e; kappa =
 *     eta = 0 is the circular orbit of Eq. (15).  The sign of the eta term
 *     is the one that the exact Keplerian orbit of Eq. (6)-(10) gives at first
 *     order in e (Eq. (11) and (14) print the opposite sign).
 */
#ifndef BSH_H
#define BSH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A cudaStream_t (NULL = legacy default stream). */
typedef struct CUstream_st* bsh_stream;

enum {
    BSH_OK = 0,
    BSH_ERR_ARG = 1,        /* bad shape, null pointer, misalignment, unsupported option */
    BSH_ERR_RANGE = 2,      /* a track leaves [k_lo, k_lo + K) or a parameter is outside the fixed-point range */
    BSH_ERR_TIMEOUT = 3,    /* a bounded device wait expired */
    BSH_ERR_CUDA = 4,       /* a CUDA runtime call failed */
    BSH_ERR_WORKSPACE = 5,  /* workspace missing or too small */
    BSH_ERR_STATE = 6       /* call order violated (e.g. plan not bound) */
};

/* Weight / accumulation dtypes. */
enum { BSH_F64 = 0, BSH_F32 = 1, BSH_F16 = 2, BSH_BF16 = 3 };

/* Number-count modes. */
enum {
    BSH_MODE_BATCHED = 0,   /* one persistent launch over every problem and patch, fixed-point
                               track with exact FP64 fallback, FP32 Kahan-compensated sums */
    BSH_MODE_PLAIN = 1,     /* one launch per sky patch, FP64 track for every term, FP64 sums */
    BSH_MODE_LUT = 2        /* BATCHED with the look-up-table approximation of Sec. IV.B in the
                               number count: in each f0 block of L = ceil(n_f0 / ceil(n_f0 / 32))
                               templates (block q: j in [qL, min(qL + L, n_f0)), length len), the
                               modulation F D is evaluated at the middle template
                               j_ref = qL + (len - 1)/2 only and reused:
                               k_j = floor(F_ref + F_ref D + 1/2) + (j - j_ref).  Stage 2
                               (bsh_power_sum) keeps the exact track. */
};

/* Text for a status code (static storage). */
const char* bsh_error_string(int status);

/* Library version: major * 10000 + minor * 100 + patch. */
int bsh_version(void);

/*
 * Reads the device status word written by kernels of this library on the
 * current device, clears it and returns it as a BSH_* code (BSH_OK when no
 * kernel reported an error).  Synchronises `stream`.  Not capturable.
 */
int bsh_sync_status(bsh_stream stream);

/* ------------------------------------------------------------------------ */
/* (i) Peakgram, Sec. IV.A, Eq. (20)-(21).                                   */
/*                                                                          */
/* power [N][K] float: SFT powers |x~|^2 of the loaded band (or, with        */
/*   median_window = 0, normalised powers rho given directly).               */
/* median_window: odd width of the running median (the paper uses 101), or   */
/*   0.  The noise floor is <n>^2 = median / ln 2 (median of Exp(1) is ln 2); */
/*   near the band edges the window is shifted, not truncated, so K must be   */
/*   >= median_window.  A row and its W words are staged in shared memory:   */
/*   with a median, (K + W) * 4 bytes must not exceed 200 KB (BSH_ERR_ARG).  */
/* rho_out [N][K] float (may be NULL): rho = P ln2 / median, rounded once    */
/*   from double.                                                             */
/* bits [N][W] uint32: bit (k & 31) of word k/32 of row i is 1 when          */
/*   P ln2 > rho_th * median (both products rounded in double), i.e.          */
/*   rho > rho_th.  W >= ceil(K/32); the padding bits are written as 0.       */
/* Capturable.                                                               */
/* ------------------------------------------------------------------------ */
int bsh_make_peakgram(const float* power, int N, int K, int median_window, double rho_th,
                      float* rho_out, uint32_t* bits, int W, bsh_stream stream);

/* ------------------------------------------------------------------------ */
/* (ii) Weights, Sec. IV.A, Eq. (22): w_i(n) = (F+^2 + Fx^2)/S_n,i at the     */
/* SFT mid-time, with F+, Fx the antenna patterns of Eq. (1).                */
/*                                                                          */
/* sky [S][3] double: unit propagation-source directions (equatorial).       */
/* arms [N][6] double: unit vectors of the x arm then the y arm of the        */
/*   detector that took SFT i, at its mid-time, same frame.                   */
/* Sn [N] double: noise level S_n of SFT i in the band (> 0).                */
/* normalize: 1 scales each sky point's weights to sum to N; 0 leaves them.  */
/* dtype: BSH_F64 / F32 / F16 / BF16, the stored type of w (round to nearest */
/*   even from the double value).                                            */
/* w [S][N] of dtype.  sum_w, sum_w2 [S] double (may be NULL): sums of the   */
/*   stored (quantised) weights and of their squares, for Eq. (25).          */
/* A sky point whose weights sum to zero records BSH_ERR_RANGE.  Capturable. */
/* ------------------------------------------------------------------------ */
int bsh_weights(const double* sky, int S, const double* arms, const double* Sn, int N,
                int normalize, int dtype, void* w, double* sum_w, double* sum_w2,
                bsh_stream stream);

/* ------------------------------------------------------------------------ */
/* Search problem: one loaded frequency band, a sky set split into patches   */
/* and a binary grid (Sec. V.A-V.B): circular orbits (a_p, Omega, t_asc), or */
/* low-eccentricity orbits with the two extra ELL1 parameters of Eq. (14).   */
/* A zero-initialised tail (n_kappa = n_eta = 0) means circular orbits.      */
/* ------------------------------------------------------------------------ */
typedef struct bsh_problem {
    /* band */
    int N;                     /* SFTs, all detectors concatenated (option B) */
    int k_lo;                  /* bin number of column 0 of the loaded band */
    int K;                     /* loaded bins per SFT */
    int W;                     /* words per peakgram row, >= ceil(K/32), multiple of 4 */
    const uint32_t* bits;      /* [N][W] peakgram from bsh_make_peakgram, 16-byte aligned */
    const float* rho;          /* [N][K] rho for stage 2, or NULL if bsh_power_sum is not used */
    const void* w;             /* [S][N] weights of w_dtype */
    int w_dtype;               /* BSH_F64 / F32 / F16 / BF16 */
    const double* sum_w;       /* [S] sum of w over SFTs */
    const double* sum_w2;      /* [S] sum of w^2 over SFTs */
    const double* v;           /* [N][3] detector velocity / c at the SFT mid-time */
    const double* t;           /* [N] SFT mid-time (s) relative to the reference time */
    double v_max;              /* bound on |v_i| (checked on the device) */
    /* frequency templates: F_j = F0 + j, j < n_f0; F0 integer or half-integer */
    double F0;
    int n_f0;
    /* sky */
    int S;
    const double* sky;         /* [S][3] unit vectors */
    int n_patch;
    const int64_t* patch_start;/* HOST [n_patch + 1]: patch p = sky points [start[p], start[p+1]) */
    /* binary grid, HOST arrays (copied by bsh_plan_create) */
    int n_ap;
    const double* a_p;         /* [n_ap] projected semi-major axis (light-seconds), >= 0 */
    int n_Om;
    const double* Omega;       /* [n_Om] orbital angular frequency 2 pi / P (rad/s), > 0 */
    int n_T;
    const double* T_asc;       /* [n_Om][n_T] time of ascension (s), Eq. (35) range */
    double rho_th;             /* peak threshold used for the peakgram (1.6), Eq. (25) mean */
    /* eccentric grid, HOST arrays (copied by bsh_plan_create); 0 / NULL = none */
    int n_kappa;
    const double* kappa;       /* [n_kappa] e cos(omega), |kappa| <= 0.5 */
    int n_eta;
    const double* eta;         /* [n_eta] e sin(omega), |eta| <= 0.5 */
    /* explicit binary bank, HOST arrays (copied by bsh_plan_create), for template banks   */
    /* whose spacing varies over the parameter space (Eq. (30)-(32)): n_orbit > 0 selects */
    /* it and the a_p / Omega / T_asc / kappa / eta grid above is not read.                */
    int n_orbit;
    const double* orbit;       /* [n_orbit][4]: Omega (> 0), t_asc, kappa, eta (|.| <= 0.5) */
    int n_bank;                /* B: binary templates, <= 2^30 */
    const int32_t* bank_orbit; /* [B] orbit row of binary template b, non-decreasing in b */
    const double* bank_ap;     /* [B] a_p of binary template b (light-seconds, >= 0) */
} bsh_problem;

typedef struct bsh_count_options {
    int mode;                  /* BSH_MODE_BATCHED, BSH_MODE_PLAIN or BSH_MODE_LUT */
    int top_k;                 /* toplist length per patch (N_C of Sec. IV.C), 1..16384 */
    int threads;               /* CTA size: 0 = autotuned / default, else 128 or 256 */
    int sft_chunk;             /* SFTs per shared-memory stage: 0 = default, else 64, 128 or 256 */
    int ctas_per_sm;           /* 0 = default; > 1 also sizes the SFT stage so that this many CTAs
                                  fit an SM's shared memory */
} bsh_count_options;

typedef struct bsh_plan bsh_plan;

/* Validates the problems on the host, picks the fixed-point scales and the
 * persistent schedule: static cost-balanced ranges of the item list, each
 * shared by a pool of CTAs (four, or two for orbit tables larger than half the
 * L2) that take its items one at a time.  HOST only, no CUDA call.  patch_start and the
 * grid or bank arrays are copied; device pointers are stored and used by later
 * calls.
 * Returns BSH_ERR_RANGE when the band does not cover every track, when a
 * parameter leaves the fixed-point range, or when a patch holds 2^32 or more
 * templates. */
int bsh_plan_create(const bsh_problem* problems, int n_problems, const bsh_count_options* opt,
                    bsh_plan** plan);
void bsh_plan_destroy(bsh_plan* plan);

/* Device workspace bytes the plan needs (tables, schedule, toplist buffers). */
size_t bsh_plan_workspace_size(const bsh_plan* plan);

/* Number of toplist regions (sum of n_patch over the problems); region r of
 * problem q is q's patch (r - first_region(q)). */
int bsh_plan_num_regions(const bsh_plan* plan);
int bsh_plan_first_region(const bsh_plan* plan, int problem);

/* Attaches the caller's workspace (256-byte aligned device memory of at least
 * bsh_plan_workspace_size bytes) and uploads the plan's small tables with
 * stream-ordered copies; synchronises `stream`.  Not capturable; call once. */
int bsh_plan_bind(bsh_plan* plan, void* workspace, size_t bytes, bsh_stream stream);

/* Runs the autotuner: times the candidate tile shapes (CTA size 256 or 128
 * binary templates, 64 / 128 / 256 SFTs per shared-memory stage, unless fixed
 * by the options; both ways of forming the binary term unless fixed by
 * bsh_plan_set_direct; per way, the two weighted-accumulation variants, or for
 * the per-term way one or two CTAs per SM) on a slice of the work list of
 * about sixteen items per CTA, best of three runs each, keeps the fastest and
 * re-uploads the plan.  Synchronises; not capturable; drops a recorded graph. */
int bsh_autotune(bsh_plan* plan, bsh_stream stream);

/* Current tile shape: CTA size, SFTs per stage, persistent CTAs in the grid. */
int bsh_plan_tile(const bsh_plan* plan, int* threads, int* sft_chunk, int* ctas);

/* Weighted-accumulation variant of the batched count:
 * 0 = one predicated FP32 add per term; 1 = per 8 SFTs a table of the 256
 * subset sums of their weights and one lookup per template.  Both sum the
 * same weights in FP32 within 4e-6 relative of their FP64 sum (Kahan
 * compensation across 64-SFT blocks) and are autotuned.  2 = on the tensor
 * cores: the 0/1 peak matrix of 2048 templates x 32 SFTs times the weights'
 * fixed-point digits round(2^24 w) in base 16 and a column of ones, in FP8
 * MMAs accumulated in FP32 without rounding, so the unweighted counts are
 * exact and the weighted counts are the exact sums of the weights' fixed-point
 * values rounded once to FP32 (fp16 weights are exact in that fixed point;
 * others differ from it by at most 2^-25 each, and a weight of 256 or more
 * records BSH_ERR_RANGE); exact-track BATCHED plans with 256-thread CTAs only
 * (BSH_ERR_ARG otherwise), one CTA per SM, not autotuned (slower on GB300).
 * bsh_plan_set_accumulate re-derives the SFT stage for the variant's
 * shared-memory layout, re-uploads a bound plan (synchronising the legacy
 * default stream) and drops a recorded graph; not capturable.  A plan that
 * forms its binary terms per term (bsh_plan_direct = 1) keeps variant 0 in
 * place of 1; there the autotuner's second candidate per shape is one CTA per
 * SM with the stage left unshrunk instead. */
int bsh_plan_set_accumulate(bsh_plan* plan, int variant);
int bsh_plan_accumulate(const bsh_plan* plan);

/* How the batched kernels form the fixed-point binary term: 0 = per warp from the staged
 * tables (the default when many templates share an orbit row), 1 = per term from the
 * thread's orbit row (the default when a warp's templates span more than 4 rows, as in
 * metric banks; the predicated-add accumulation is then used), -1 = automatic.  Rebuilds
 * the schedule like bsh_plan_set_accumulate; not capturable.  bsh_plan_direct returns the
 * choice in effect. */
int bsh_plan_set_direct(bsh_plan* plan, int mode);
int bsh_plan_direct(const bsh_plan* plan);

/* Bounded waits of the batched count.  Each CTA stages SFT chunks through two
 * buffers and waits on a barrier per stage; a wait polls at most `polls` times
 * (0 = the default, 2^22 polls: about a second or more) and then gives up: the
 * CTA waits, with the same bound, for the copies it still has in flight, frees
 * its tensor memory and exits, and bsh_sync_status returns BSH_ERR_TIMEOUT.
 * skip_stage is a test hook for that path: >= 0 makes every CTA leave the copies
 * of its skip_stage-th stage (0 = its first) unissued, so that the wait on them
 * expires without any fault; -1 (the default) issues every stage.  Drops a
 * recorded graph; not capturable.  The paper has no counterpart: this is the
 * library's own failure detection. */
int bsh_plan_set_wait(bsh_plan* plan, int polls, int skip_stage);

/* ------------------------------------------------------------------------ */
/* (iii) Number count, Sec. IV.C and V.A: for every template the weighted    */
/* sum n = sum_i w_i * bit_i[k_i] along the track k_i = round(f(t_i) T_c) of  */
/* Eq. (14)/(15), its significance s_H of Eq. (25), and a fused per-patch    */
/* toplist of the top_k largest s_H (ties: smaller template id first).       */
/* Reads the problems' bits, w, sums, v, t and sky arrays.  Capturable.      */
/* The batched kernels keep their running sums in tensor memory: each CTA    */
/* takes half a column per thread (at most 256 of an SM's 512 columns) and   */
/* frees them before it exits; a CTA that starts while other work on its SM  */
/* holds the columns it needs waits until they are freed.                    */
/* ------------------------------------------------------------------------ */
int bsh_number_count(bsh_plan* plan, bsh_stream stream);

/* Debug / parity form of (iii): writes every template's counts instead of a
 * toplist.  n_unw[q] and n_w[q] are HOST arrays of n_problems DEVICE pointers
 * to [S][B][n_f0] int32 / float buffers.  Capturable. */
int bsh_count_dense(bsh_plan* plan, int32_t* const* n_unw, float* const* n_w, bsh_stream stream);

/* ------------------------------------------------------------------------ */
/* (iv) Toplist, Sec. IV.C: merges the per-CTA candidate lists of each        */
/* region into its top_k templates, sorted by s_H (descending, ties by       */
/* template id).                                                              */
/* out [regions][top_k]; n_out [regions] entries written.  Capturable.       */
/* ------------------------------------------------------------------------ */
typedef struct bsh_cand {
    int64_t template_id;       /* ((s * B + b) * n_f0 + j) within the problem */
    float s_h;                 /* Eq. (25) */
    float n_w;                 /* weighted number count */
    int32_t n_unw;             /* unweighted number count */
    float power;               /* Eq. (26) P, set by bsh_power_sum */
    float s_p;                 /* Eq. (26) s_P, set by bsh_power_sum */
    int32_t region;            /* toplist region (problem's first region + patch) */
} bsh_cand;

int bsh_toplist(bsh_plan* plan, bsh_cand* out, int32_t* n_out, bsh_stream stream);

/* ------------------------------------------------------------------------ */
/* (v) Stage 2, Sec. IV.C, Eq. (26): for every candidate the summed weighted  */
/* normalised power P = sum_i w_i rho_i[k_i] along the exact track, and       */
/* s_P = (P - sum w)/sqrt(sum w^2); then each region's list is re-ranked by  */
/* s_P (descending, ties by template id) and cut to n_cf (N_CF).             */
/* cands [regions][top_k] and n_cands [regions] as written by bsh_toplist     */
/* (power and s_p are filled in place); final [regions][n_cf], n_final       */
/* [regions].  Needs every problem's rho.  Capturable.                        */
/* ------------------------------------------------------------------------ */
int bsh_power_sum(bsh_plan* plan, bsh_cand* cands, const int32_t* n_cands, int n_cf,
                  bsh_cand* final_list, int32_t* n_final, bsh_stream stream);

/* ------------------------------------------------------------------------ */
/* (v') Stage 2 on another SFT set, Sec. IV.C: the power sums of Eq. (26) of */
/* plan `stage1`'s candidate lists computed with the SFTs of plan `stage2`   */
/* -- the stage-1 SFTs together with the complementary SFTs that start T_c/2 */
/* later (where T_c contiguous seconds of data exist), about twice as many.  */
/* stage2's problems must search the same templates as stage1's (same sky    */
/* points in the same patches, binary templates, F0 and n_f0; checked on the */
/* host except for the sky values) and carry rho.  cands / n_cands as written */
/* by bsh_toplist on stage1 (stride stage1's top_k); n_cf <= stage1's top_k; */
/* final_list [regions][n_cf], n_final [regions] as for bsh_power_sum.      */
/* stage2 is a BATCHED plan that needs no bsh_number_count: its track tables */
/* are computed here.  Capturable.                                           */
/* ------------------------------------------------------------------------ */
int bsh_power_sum_sft(bsh_plan* stage2, const bsh_plan* stage1, bsh_cand* cands, const int32_t* n_cands, int n_cf,
                      bsh_cand* final_list, int32_t* n_final, bsh_stream stream);

/* ------------------------------------------------------------------------ */
/* CUDA-graph form of (iii)+(iv)+(v): the first call records the three calls */
/* on `stream` into a graph owned by the plan, later calls replay it.         */
/* Arguments as for bsh_toplist and bsh_power_sum; changing them requires     */
/* bsh_graph_reset.  Not capturable itself.                                   */
/* ------------------------------------------------------------------------ */
int bsh_graph_launch(bsh_plan* plan, bsh_cand* cands, int32_t* n_cands, int n_cf,
                     bsh_cand* final_list, int32_t* n_final, bsh_stream stream);
int bsh_graph_reset(bsh_plan* plan);

/* ------------------------------------------------------------------------ */
/* Track diagnostics, Eq. (14)/(15).                                         */
/* bsh_track_precision: for every term of sky points [s_begin, s_end) of the */
/* plan's problem (every binary template, SFT and f0 template) compares the  */
/* exact FP64 bin with (a) the same expression evaluated in single          */
/* precision and (b) the fixed-point bin of the batched kernels.  counts [4] */
/* DEVICE uint64: terms, single-precision mismatches, fixed-point mismatches */
/* outside the tie band, terms inside the 1e-9-bin tie band.  Capturable.    */
/* bsh_track_bins: exact bins of listed templates (ids as in bsh_cand) in   */
/* every SFT: bins [n][N] DEVICE int32 (bin numbers, not band columns), e.g. */
/* to place injected signals.  Capturable.                                   */
/* ------------------------------------------------------------------------ */
int bsh_track_precision(bsh_plan* plan, int problem, int s_begin, int s_end, unsigned long long* counts,
                        bsh_stream stream);
int bsh_track_bins(bsh_plan* plan, int problem, const int64_t* ids, int n, int32_t* bins, bsh_stream stream);

/* ------------------------------------------------------------------------ */
/* Host-side checks of the fixed-point track (no GPU needed).                 */
/* Evaluates, on the host with the same code as the kernels, the 32-bit       */
/* peak window of templates (s, b, block j0..j0+31) at SFT i for `count`      */
/* queries: row_bits [count][W] holds the row of each query; out [count]     */
/* receives the windows and path [count] the path taken (0 fast, 1 crossing,  */
/* 2 exact-fallback).  Inputs as in bsh_problem but HOST arrays.  Used by the */
/* CPU tests against the oracle.                                              */
/* ------------------------------------------------------------------------ */
int bsh_debug_track_windows(const bsh_problem* host_problem, const int32_t* query /*[count][4]: s,b,i,j0*/,
                            int count, const uint32_t* row_bits, uint32_t* out, int32_t* path);

/* ------------------------------------------------------------------------ */
/* Host-side view of the batched schedule (no GPU needed; no counterpart in  */
/* the paper: the order of work is this library's).  The batched kernels'   */
/* CTAs share the item list in pools: pool q is a contiguous, cost-balanced  */
/* range of items that its CTAs (pool_size of them) take one at a time, in   */
/* the pool's walk order.  Items of a problem run sky point, binary tile,    */
/* f0 block (fastest); indices count from the first problem's first item.    */
/* *n_pools and *pool_size receive the plan's counts (either may be NULL);   */
/* for 0 <= pool < n_pools, *n_items (may be NULL) receives the pool's item  */
/* count and, when items is not NULL and cap >= that count, items[] its walk */
/* order.  BATCHED and LUT plans only (BSH_ERR_STATE otherwise); pool out of */
/* range or cap too small: BSH_ERR_ARG.  The schedule is the one that        */
/* bsh_plan_create, or the last bsh_autotune, left.                          */
/* ------------------------------------------------------------------------ */
int bsh_debug_pool_walk(const bsh_plan* plan, int pool, int64_t* items, int64_t cap, int64_t* n_items,
                        int* n_pools, int* pool_size);

/* ------------------------------------------------------------------------ */
/* (vi) Post-processing, Sec. V.E: candidate parameters, the distance of      */
/* Eq. (44), coincidences between two lists (option A), clustering, the       */
/* option-B cut, significance-weighted centroids and each band's most         */
/* significant cluster.                                                       */
/*                                                                          */
/* Parameters of a candidate: (f in Hz, x, y, a_p, Omega, t_asc), x and y the */
/* sky direction in ecliptic Cartesian coordinates projected on the ecliptic  */
/* plane (x = n_x, y = cos(obliquity) n_y + sin(obliquity) n_z).  Distance:   */
/*   d^2 = sum over the six parameters of (difference / resolution)^2,        */
/* each resolution the mean of its values at the two candidates: delta f =   */
/* 1/T_c; delta theta = 1/(v_over_c T_c f P_F) for x and y; delta a_p, delta  */
/* Omega, delta t_asc of Eq. (30)-(32).  Thresholds are strict (d < d_cluster,*/
/* d < d_coinc); the cut keeps d <= d_cut.  Centroid weights are max(sig, 0), */
/* the plain mean where they sum to 0.  FP64 throughout, each operation       */
/* rounded separately.                                                        */
/* ------------------------------------------------------------------------ */
typedef struct bsh_post_params {
    double T_c;                /* coherence time (s): f = F / T_c, delta f = 1 / T_c */
    double T_obs;              /* observation time (s), Eq. (31) */
    double v_over_c;           /* detector speed / c in delta theta (Sec. V.B) */
    double P_F;                /* pixel factor of delta theta */
    double m_a, m_Om, m_t;     /* mismatch parameters of Eq. (30)-(32) */
    double obliquity;          /* rad, equatorial -> ecliptic rotation about x */
    double d_cluster;          /* clustering threshold (bins; sqrt(14) in Sec. VI) */
    double d_cut;              /* option-B cut around each cluster's top member (bins); <= 0: none */
    double d_coinc;            /* coincidence threshold (bins; 3 in Sec. VI) */
} bsh_post_params;

/* Parameters of problem `problem`'s candidates: region r = first_region + p  */
/* (patch p), rank e < per_region give row n = p * per_region + e of params   */
/* [n][6] and sig [n] (s_H with stat 0, s_P with stat 1) as doubles; valid [n] */
/* = e < n_cands[r].  cands [regions][per_region], n_cands [regions]: the     */
/* lists of bsh_toplist (per_region = top_k) or bsh_power_sum's final lists   */
/* (per_region = n_cf).  All DEVICE.  Capturable.                            */
int bsh_cand_params(bsh_plan* plan, int problem, const bsh_cand* cands, const int32_t* n_cands, int per_region,
                    int stat, const bsh_post_params* pp, double* params, double* sig, int32_t* valid,
                    bsh_stream stream);

/* Workspace bytes of bsh_cluster for n candidates. */
size_t bsh_cluster_workspace(int n);

/* Clusters one band's n <= 2^20 candidates (DEVICE arrays): label [n] = the  */
/* smallest index of the candidate's connected component (edges between valid */
/* candidates with d < d_cluster), -1 where valid[i] = 0; keep [n] = 1 for    */
/* members within d_cut of their cluster's top member (largest sig, then the  */
/* smallest index); centroid [n][6] and csig [n] at each root's row (label[i] */
/* == i): the weighted mean and the summed sig of the kept members (NaN and 0 */
/* at the other rows); best [1] = the root with the largest csig (ties: the   */
/* smallest root), -1 if there is none.  work: bsh_cluster_workspace(n)       */
/* bytes of DEVICE memory.  Capturable.                                      */
int bsh_cluster(const double* params, const double* sig, const int32_t* valid, int n, const bsh_post_params* pp,
                void* work, size_t work_bytes, int32_t* label, int32_t* keep, double* centroid, double* csig,
                int32_t* best, bsh_stream stream);

/* Workspace bytes of bsh_coincidences. */
size_t bsh_coincidence_workspace(int na, int nb);

/* Option A: every pair (i of list A, j of list B, both valid) with d <       */
/* d_coinc, in an unspecified order: pairs [cap][2] = (i, j), centroid        */
/* [cap][6] and sig [cap] = sa[i] + sb[j]; n_pairs [1] = the number of pairs  */
/* found (entries past cap are not written).  DEVICE arrays; na, nb <= 2^20.  */
/* Capturable.                                                                */
int bsh_coincidences(const double* pa, const double* sa, const int32_t* va, int na, const double* pb,
                     const double* sb, const int32_t* vb, int nb, const bsh_post_params* pp, void* work,
                     size_t work_bytes, int32_t* pairs, double* centroid, double* sig, int cap, int32_t* n_pairs,
                     bsh_stream stream);

/* ------------------------------------------------------------------------ */
/* Binary template bank, Sec. V.B, Eq. (30)-(32).  HOST only, no CUDA call.   */
/*                                                                          */
/* bsh_binary_resolution: the spacings at (f, a_p, Omega) for the mismatch   */
/*   parameters m_a, m_Om, m_t (f in Hz, T_c and T_obs in s, a_p in          */
/*   light-seconds, Omega in rad/s):                                         */
/*     d_ap = sqrt(6 m_a) / (pi T_c f Omega)                                 */
/*     d_Om = sqrt(72 m_Om) / (pi T_c f a_p Omega T_obs)                     */
/*     d_t  = sqrt(6 m_t) / (pi T_c f a_p Omega^2)                           */
/* bsh_template_bank: a bank over a_p in [ap_min, ap_max], P in [P_min,       */
/*   P_max] and t_asc within half a period of t_mid (Eq. (35)), as orbit rows */
/*   and (row, a_p) entries in the layout of bsh_problem's explicit bank:     */
/*   Omega from 2 pi / P_max upwards, each step d_Om at ap_max, until past    */
/*   2 pi / P_min; at each Omega, a_p from ap_min in steps of d_ap(Omega)     */
/*   up to ap_max, cut into blocks whose largest / smallest a_p ratio is at   */
/*   most ap_block; each block gets t_asc values from t_mid - P/2 in steps of */
/*   d_t at the block's largest a_p, below t_mid + P/2.  Every spacing is the */
/*   smallest the metric asks for over the cell it covers.  Call with NULL    */
/*   arrays for the sizes (n_orbit, n_bank), then with arrays of at least     */
/*   those capacities; BSH_ERR_WORKSPACE if a capacity is too small,          */
/*   BSH_ERR_RANGE if P_min <= T_c or the bank would exceed 2^30 entries.     */
/* ------------------------------------------------------------------------ */
typedef struct bsh_bank_spec {
    double f;                  /* frequency (Hz) the spacings use: the band's highest */
    double T_c, T_obs;         /* coherence time and observation time (s) */
    double t_mid;              /* centre of the t_asc range (s) */
    double ap_min, ap_max;     /* light-seconds, 0 < ap_min <= ap_max */
    double P_min, P_max;       /* orbital period (s), T_c < P_min <= P_max */
    double m_a, m_Om, m_t;     /* mismatch parameters (> 0) */
    double ap_block;           /* a_p ratio sharing one t_asc grid (>= 1) */
} bsh_bank_spec;

int bsh_binary_resolution(double f, double T_c, double T_obs, double a_p, double Omega, double m_a, double m_Om,
                          double m_t, double* d_ap, double* d_Om, double* d_t);
int bsh_template_bank(const bsh_bank_spec* spec, int* n_orbit, double* orbit, int orbit_cap, int* n_bank,
                      int32_t* bank_orbit, double* bank_ap, int bank_cap);

/* ------------------------------------------------------------------------ */
/* Stage-2 power sum that allocates nothing.  The paper has no counterpart:  */
/* this entry point exists for callers that cannot allocate device memory   */
/* (for example code running where cudaMalloc is forbidden or unavailable,  */
/* such as inside a host callback, a memory-pool-less embedding, or a        */
/* process whose allocator is owned by another runtime).  It needs no plan  */
/* and no workspace: its scratch (the FP64 / fixed-point track tables and   */
/* weights of one problem) lives in one static device array of              */
/* BSH_STATIC_SCRATCH_BYTES that every GPU loading this library keeps until */
/* process exit.                                                              */
/*                                                                          */
/* problem: as for bsh_plan_create (HOST grid and patch arrays, DEVICE data */
/*   arrays, rho required).  template_ids [n] DEVICE int64:                  */
/*   template ids ((s * B + b) * n_f0 + j).  power, s_p [n] DEVICE float:     */
/*   P and s_P of Eq. (26) for each id, the same values bsh_power_sum gives. */
/* Returns BSH_ERR_WORKSPACE when the problem's tables exceed the static     */
/* array: S * N' * 8 + R * N' * 12 + B * 16 bytes plus the grids, with N' = */
/* N rounded up to 256, R the orbit rows (n_Om * n_T * max(1, n_kappa) *    */
/* max(1, n_eta) for a grid, n_orbit for a bank) and B the binary templates.*/
/* The first call on a device looks up the array's device address (make    */
/* that first call before any stream capture).  Every call overwrites the   */
/* whole array, so calls that overlap on the GPU (other streams, other      */
/* threads) race and must be serialised by the caller.                      */
/* Kernel-side errors are reported by bsh_sync_status.                      */
/* ------------------------------------------------------------------------ */
#define BSH_STATIC_SCRATCH_BYTES (32u << 20)
int bsh_power_sum_static(const bsh_problem* problem, const int64_t* template_ids, int n, float* power,
                         float* s_p, bsh_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* BSH_H */
