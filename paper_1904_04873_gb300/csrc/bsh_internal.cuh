// Internal declarations shared by the CUDA translation units of libbsh.
//
// Track arithmetic (Eq. (14)/(15) times T_c):
//   k_i(j) = floor(F_j + F_j * D_i + 1/2),  D_i = v_i.n - a_p * (Omega * g_i),
//   g_i = (cos(phi) + kappa cos(2 phi)) + eta sin(2 phi),  phi = Omega (t_i - t_asc)
// (kappa = eta = 0: circular orbit, g_i = cos(phi)).
// The hot kernels evaluate it in 32-bit fixed point, with a rigorous error
// bound eps, and fall back to the exact FP64 expression whenever the fixed-point
// value lies within M > eps of a rounding boundary.  The fixed-point value of
//   v(j) = F_j * D + frac(F_j) + 1/2        (units of bins, scale 2^s_y)
// is Z(j) - mulhi(ap_q, C_q(j)) with
//   Z(j)   = round(F_j * vn * 2^s_y) + (frac(F_j) + 1/2) 2^s_y    from vn_q = round(vn 2^s_vn)
//   C_q(j) = round(F_j * c * 2^s_C)                               from c_q  = round(c 2^s_c), c = Omega g
//   ap_q   = round(a_p 2^s_a),  s_y = s_a + s_C - 32
// and the bin is floor(F_j) + floor(v(j) / 2^s_y).  The exact value is linear in
// j with slope D 2^s_y, so a block of 32 consecutive f0 templates [j0, j0 + 31]
// reads one 32-bit window when v at the reference template j0 + 15, widened by
// the margin mg = 16 |D|max 2^s_y + M, stays inside one cell; |D|max is bounded
// per SFT from vn_q and the problem's a_p Omega bound (fp_margin).  Otherwise the
// (block, SFT) pair is deferred to the end of its SFT chunk, where v is evaluated
// at both ends of the block (fp_window_ends, then fp_window_exact per template).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/bsh.h"

#ifndef __CUDACC__
#define __host__
#define __device__
#define __forceinline__ inline
#endif

namespace bsh {

constexpr int MAX_PROBLEMS = 8;
constexpr int JW = 32;            // f0 templates per thread (one 32-bit peak window)

// Device status word bits (reported as the lowest set code by bsh_sync_status).
enum : unsigned {
    ST_RANGE = 1u << 0,
    ST_TIMEOUT = 1u << 1,
    ST_ARG = 1u << 2,
};

__device__ __forceinline__ void set_status(unsigned* status, unsigned bit) {
#ifdef __CUDA_ARCH__
    atomicOr(status, bit);
#else
    *status |= bit;
#endif
}

// Fixed-point parameters of one problem (chosen on the host, see plan.cu).
struct FixedPoint {
    int s_vn, s_c, s_a, s_C, s_y;
    int sh_v, sh_c;               // right shifts producing Z and C_q from the tables
    int M;                        // decision margin (units of 2^-s_y bins)
    int off_q;                    // (frac(F0) + 1/2) 2^s_y
    double eps;                   // error bound of v (units of 2^-s_y bins)
    int mg_a;                     // 16 a_p,max |c|max 2^s_y + M + 2: binary part of the slope margin
    int mg_k;                     // (|vn_q| + 2^mg_k) >> mg_k >= 16 |vn| 2^s_y (vn part of the margin)
};

// Per-problem data seen by the kernels.
struct ProbDev {
    // caller arrays
    const uint32_t* bits;     // [N][W]
    const float* rho;         // [N][K]
    const void* w;            // [S][N] (w_dtype)
    const double* sum_w;      // [S]
    const double* sum_w2;     // [S]
    const double* v;          // [N][3]
    const double* t;          // [N]
    const double* sky;        // [S][3]
    // workspace tables
    int32_t* vn_q;            // [S][Np]
    int32_t* c_q;             // [nOT][Np]   one row per orbit (Omega, t_asc, kappa, eta)
    double* c64;              // [nOT][Np]
    float* w32;               // [S][Np]   (batched mode)
    double* w64;              // [S][Np]   (plain mode)
    // binary templates: orbit rows and, per template b, its row, a_p and fixed-point a_p
    const double* orb;        // [nOT][4] Omega, t_asc, kappa, eta
    const int32_t* brow;      // [B] orbit row of template b (non-decreasing in b)
    const double* bap;        // [B] a_p of template b
    const int32_t* bapq;      // [B] round(a_p 2^s_a)
    const int64_t* patch_start;  // [n_patch + 1]
    const int32_t* patch_of_s;   // [S]
    // sizes
    int N, Np, K, W, k_lo, n_f0, S, nOT, B, n_patch, w_dtype;
    double F0;                // first template (bins)
    int G0;                   // floor(F0)
    int JB;                   // valid templates per f0 block (<= 32)
    int n_fb, n_bt;           // f0 blocks, binary tiles
    int crows;                // orbit rows per staged box of c_q (batched mode)
    FixedPoint fp;
    int o_min, o_max;         // bounds of floor(v / 2^s_y)
    int Wseg;                 // staged words per row
    double p_th;              // exp(-rho_th)
    double v_max;
    int region_base;
    int64_t item_begin, n_items;
    int64_t cost;             // cost units per item
};

// Entry of a toplist buffer: key = (order-preserving bits of s_H) << 32 | (2^32 - 1 - local id).
struct Entry {
    unsigned long long key;
    float n_w;
    int32_t n_unw;
};
static_assert(sizeof(Entry) == 16, "Entry layout");

__host__ __device__ __forceinline__ uint32_t float_order(float f) {
    uint32_t u;
#ifdef __CUDA_ARCH__
    u = __float_as_uint(f);
#else
    union { float f; uint32_t u; } cv;
    cv.f = f;
    u = cv.u;
#endif
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__host__ __device__ __forceinline__ float order_float(uint32_t o) {
    uint32_t u = (o & 0x80000000u) ? (o & 0x7fffffffu) : ~o;
#ifdef __CUDA_ARCH__
    return __uint_as_float(u);
#else
    union { float f; uint32_t u; } cv;
    cv.u = u;
    return cv.f;
#endif
}

__host__ __device__ __forceinline__ unsigned long long make_key(float score, uint32_t lid) {
    return ((unsigned long long)float_order(score) << 32) | (unsigned long long)(0xffffffffu - lid);
}

__host__ __device__ __forceinline__ int mulhi32(int a, int b) {
#ifdef __CUDA_ARCH__
    return __mulhi(a, b);
#else
    return (int)(((long long)a * (long long)b) >> 32);
#endif
}

__host__ __device__ __forceinline__ int imin(int a, int b) { return a < b ? a : b; }
__host__ __device__ __forceinline__ int imax(int a, int b) { return a > b ? a : b; }

// Z(j) from a vn table entry: round(F2 * vn_q / 2^sh_v) + off_q, F2 = 2 F_j.
__host__ __device__ __forceinline__ int make_Z(int F2, int vn_q, const FixedPoint& fp) {
    long long p = (long long)F2 * (long long)vn_q;
    long long r = fp.sh_v > 0 ? ((p + (1LL << (fp.sh_v - 1))) >> fp.sh_v) : p;
    return (int)r + fp.off_q;
}

// C_q(j) from a c table entry: round(F2 * c_q / 2^sh_c).
__host__ __device__ __forceinline__ int make_C(int F2, int c_q, const FixedPoint& fp) {
    long long p = (long long)F2 * (long long)c_q;
    long long r = fp.sh_c > 0 ? ((p + (1LL << (fp.sh_c - 1))) >> fp.sh_c) : p;
    return (int)r;
}

// Margin of the reference-template test for an SFT with table entry vn_q.
__host__ __device__ __forceinline__ int fp_margin(int vn_q, const FixedPoint& fp) {
    const unsigned a = (unsigned)(vn_q < 0 ? -vn_q : vn_q);
    return fp.mg_a + (int)((a + (1u << fp.mg_k)) >> fp.mg_k);
}

// Reference-template test: v widened by mg on both sides stays in one cell.
__host__ __device__ __forceinline__ bool fp_fast_ref(int v, int mg, int s_y) {
    return ((unsigned)((v - mg) ^ (v + mg)) >> s_y) == 0u;
}

// 32 consecutive bits of a staged row starting at bit position pos (0 <= pos <= 32*Wseg - 33).
__host__ __device__ __forceinline__ uint32_t row_window(const uint32_t* row, int pos) {
    uint32_t w0 = row[pos >> 5], w1 = row[(pos >> 5) + 1];
#ifdef __CUDA_ARCH__
    return __funnelshift_r(w0, w1, pos & 31);
#else
    int sh = pos & 31;
    return sh ? ((w0 >> sh) | (w1 << (32 - sh))) : w0;
#endif
}

__host__ __device__ __forceinline__ uint32_t row_bit(const uint32_t* row, int pos) {
    return (row[pos >> 5] >> (pos & 31)) & 1u;
}

// Two-ended test of a block whose reference-template test failed.  V_j = 31 v0 + d j
// (d = v1 - v0) is 31 v(j) exactly interpolated.  Path 0: both ends, widened by M,
// in one cell.  Path 1: the ends in adjacent cells and a single crossing at least
// 31 M from every template point: templates below the crossing read the first cell,
// the others the second.  Returns false (path 2) when neither holds; the caller then
// decides template by template (fp_window_exact).
__host__ __device__ __forceinline__ bool fp_window_ends(int v0, int v1, int pbase, int pos_max, int s, int M,
                                                        const uint32_t* row, uint32_t* out, int* path) {
    const int vmin = imin(v0, v1), vmax = imax(v0, v1);
    const int ca = vmin >> s, cb = vmax >> s;
    if (((unsigned)((vmin - M) ^ (vmax + M)) >> s) == 0u) {
        const int p0 = pbase + ca;
        if ((unsigned)p0 > (unsigned)pos_max) return false;
        *path = 0;
        *out = row_window(row, p0);
        return true;
    }
    if (cb != ca + 1) return false;
    const long long lo_edge = (long long)ca << s, Bc = (long long)cb << s, hi_edge = ((long long)cb + 1) << s;
    if ((long long)vmin - lo_edge < M || hi_edge - (long long)vmax < M) return false;
    const long long d = (long long)v1 - (long long)v0;       // nonzero: the ends are in different cells
    const long long B31 = 31LL * Bc, V0 = 31LL * v0;
    // jc = first j with V_j on the far side of 31 Bc; estimated in single precision
    // (error below one step) and settled with exact integer comparisons
    // (32-bit operands: Bc - v0 and v1 - v0 lie within two cells, |.| < 2^31)
    const float est = (31.0f * (float)((int)Bc - v0)) / (float)(v1 - v0);
    int jc = (int)ceilf(est);
    jc = jc < 0 ? 0 : (jc > 32 ? 32 : jc);
    for (int it = 0; it < 2; ++it) {
        const bool far_jc = d > 0 ? (V0 + d * jc >= B31) : (V0 + d * jc < B31);
        const bool far_prev = jc > 0 && (d > 0 ? (V0 + d * (jc - 1) >= B31) : (V0 + d * (jc - 1) < B31));
        if (far_prev) --jc;
        else if (!far_jc && jc < 32) ++jc;
        else break;
    }
    if (jc < 1 || jc > 31) return false;
    const long long Vm = V0 + d * (jc - 1), Vp = V0 + d * jc;
    const bool ok_m = d > 0 ? (Vm < B31) : (Vm >= B31);
    const bool ok_p = d > 0 ? (Vp >= B31) : (Vp < B31);
    const long long M31 = 31LL * M;
    const long long dm = Vm > B31 ? Vm - B31 : B31 - Vm;
    const long long dp = Vp > B31 ? Vp - B31 : B31 - Vp;
    if (!ok_m || !ok_p || dm < M31 || dp < M31) return false;
    const int o0 = v0 >> s;
    const int o1 = d > 0 ? o0 + 1 : o0 - 1;
    const int p0 = pbase + o0, p1 = pbase + o1;
    if ((unsigned)p0 > (unsigned)pos_max || (unsigned)p1 > (unsigned)pos_max) return false;
    const uint32_t low = (1u << jc) - 1u;
    *path = 1;
    *out = (row_window(row, p0) & low) | (row_window(row, p1) & ~low);
    return true;
}

// Path 2: each template's cell from V_j when it is at least 31 M from a boundary, else
// by the exact FP64 expression (exact_o(j) returns floor(F_j + F_j D + 1/2) - floor(F_j)).
// Bits whose position falls outside the staged row set *bad and read as 0.
template <class ExactO>
__host__ __device__ uint32_t fp_window_exact(int v0, int v1, int pbase, int pos_max, int s, int M,
                                             const uint32_t* row, ExactO exact_o, bool* bad) {
    const long long d = (long long)v1 - (long long)v0;
    const long long S31 = 31LL << s;
    const long long M31 = 31LL * M;
    const int ca = imin(v0, v1) >> s;
    uint32_t m = 0;
    const long long base = 31LL * ((long long)ca << s);
    for (int j = 0; j < 32; ++j) {
        const long long V = 31LL * v0 + d * j;
        long long rel = V - base;                 // >= 0
        int q = ca;
        while (rel >= S31) { rel -= S31; ++q; }
        int o;
        if (rel < M31 || rel > S31 - M31) o = exact_o(j);
        else o = q;
        const int pos = pbase + j + o;
        if (pos < 0 || pos >= pos_max + 33) { *bad = true; continue; }
        m |= row_bit(row, pos) << j;
    }
    return m;
}

// Both together (host checks and the plain tools): path 0, 1 or 2.
template <class ExactO>
__host__ __device__ uint32_t fp_window_slow(int v0, int v1, int pbase, int pos_max, int s,
                                            int M, const uint32_t* row, ExactO exact_o,
                                            int* path, bool* bad) {
    uint32_t m = 0;
    if (fp_window_ends(v0, v1, pbase, pos_max, s, M, row, &m, path)) return m;
    *path = 2;
    return fp_window_exact(v0, v1, pbase, pos_max, s, M, row, exact_o, bad);
}

#ifdef __CUDACC__
// Stage 2, Eq. (26), for one template (s, b, j): P = sum_i w_i rho_i[k_i] along its exact
// track, one warp with lanes over SFTs.  The bin of each term is the fixed-point track's,
// or the FP64 expression within the margin M of a rounding boundary.  FP32 weights: a
// Kahan-compensated FP32 sum per lane, then a shuffle tree; FP64 weights (the plain form):
// FP64 sums.  Every lane returns the total.  A bin outside the loaded band records ST_RANGE
// and its term is skipped.
__device__ __forceinline__ double warp_power_sum(const ProbDev& P, int s, int b, int j, unsigned* status) {
    const int lane = threadIdx.x & 31;
    const double F = P.F0 + (double)j;
    const int F2 = (int)llrint(2.0 * F);
    const int G = P.G0 + j;
    const int ot = P.brow[b];
    const int apq = P.bapq[b];
    const double ap = P.bap[b];
    const int s_y = P.fp.s_y, M = P.fp.M;
    const int cell = 1 << s_y;
    const bool plain = P.w64 != nullptr && P.w32 == nullptr;
    const double* n = P.sky + 3 * (size_t)s;
    float sum = 0.f, comp = 0.f;
    double sum64 = 0.0;
    for (int i = lane; i < P.N; i += 32) {
        const int Z = make_Z(F2, P.vn_q[(size_t)s * P.Np + i], P.fp);
        const int C = make_C(F2, P.c_q[(size_t)ot * P.Np + i], P.fp);
        const int v = Z - mulhi32(apq, C);
        const int fr = v & (cell - 1);
        int o = v >> s_y;
        if (fr < M || fr > cell - M) {
            const double* vv = P.v + 3 * (size_t)i;
            const double vn = __dadd_rn(__dadd_rn(__dmul_rn(vv[0], n[0]), __dmul_rn(vv[1], n[1])),
                                        __dmul_rn(vv[2], n[2]));
            const double D = __dsub_rn(vn, __dmul_rn(ap, P.c64[(size_t)ot * P.Np + i]));
            const double x = __dadd_rn(F, __dmul_rn(F, D));
            o = (int)((long long)floor(__dadd_rn(x, 0.5)) - (long long)G);
        }
        const int col = G + o - P.k_lo;
        if (col < 0 || col >= P.K) {
            set_status(status, ST_RANGE);
            continue;
        }
        const float rho = __ldg(P.rho + (size_t)i * P.K + col);
        if (plain) {
            sum64 = __dadd_rn(sum64, __dmul_rn(P.w64[(size_t)s * P.Np + i], (double)rho));
        } else {
            const float x = P.w32[(size_t)s * P.Np + i] * rho;
            const float y = x - comp;
            const float t = sum + y;
            comp = (t - sum) - y;
            sum = t;
        }
    }
    if (plain) {
        for (int o = 16; o > 0; o >>= 1) sum64 += __shfl_xor_sync(0xffffffffu, sum64, o);
        return sum64;
    }
    float v = sum - comp;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return (double)v;
}
#endif

// Raises a kernel's dynamic shared-memory limit once (never inside a graph
// capture once the first eager launch has set it).
template <class K>
inline void ensure_smem(K kernel, int bytes, int* done) {
    if (bytes > *done) {
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        *done = bytes;
    }
}

// ---------------------------------------------------------------- launches
// CTAs per item pool of the batched kernels at most: two SMs' worth, each SM holding one CTA
// that its warp schedulers favour and one that they do not
constexpr int kPoolMax = 4;

struct CountArgs {
    const ProbDev* probs;        // device array [n_probs]
    int n_probs;
    const int64_t* cta_item;     // [ctas + 1] item range per CTA (plain kernel)
    const int32_t* cta_visit;    // [ctas] first visit index per CTA (plain kernel)
    // batched kernels: CTAs c + m * pools (m < pool_size) share pool c (c < pools)
    int pools;
    int pool_size;               // CTAs per pool (2 or kPoolMax)
    const int64_t* pool_item;    // [pools + 1] item range of each pool
    const int32_t* pool_sweep;   // [2 * pools] walk of each pool: rotation r, sweep length P
    const int32_t* pool_run;     // [pools + 1] each pool's runs (one region along its walk) in run_step
    const int64_t* run_step;     // [runs] first walk step of each run; run j owns visits pool_size j + m
    unsigned long long* pool_next;  // [pools] next walk step of each pool (zeroed before each launch)
    Entry* visit_buf;            // [visits][cap]
    int32_t* visit_count;        // [visits]
    int cap;                     // entries per visit buffer
    int top_k;
    int dense;                   // write dense counts instead of toplists
    int32_t* const* dense_unw;   // device array [n_probs] of device pointers
    float* const* dense_w;
    unsigned* status;
    int chunk;                   // SFTs per stage
    int smem_bytes;
    int wseg_max, ot_max;
    int mode;                    // BSH_MODE_*
    int max_n;                   // largest SFT count of the problems
    int wrows;                   // Omega-T rows one warp needs at most
    int acc_mode;                // weighted accumulation: 0 predicated adds, 1 byte table, 2 tensor cores
    int lut;                     // 1: look-up-table approximation of the track (BSH_MODE_LUT)
    int direct;                  // 1: C_q formed per term from the staged rows (predicated-add only)
    int wait_polls;              // polls of a staging barrier before a wait gives up (BSH_ERR_TIMEOUT)
    int skip_stage;              // test hook: per-CTA stage sequence number left unissued (-1: none)
};

// TMA descriptors of the batched kernel, one pair per problem: the peakgram rows and
// the fixed-point orbit table c_q.
struct TmapSet {
    alignas(64) unsigned char map[MAX_PROBLEMS][128];
    alignas(64) unsigned char cmap[MAX_PROBLEMS][128];
};

void launch_count(const CountArgs& a, const TmapSet& maps, int grid, int threads, cudaStream_t st);
// tensor-core accumulation of the batched count (acc_mode 2; count_tc.cu)
void launch_count_tc(const CountArgs& a, const TmapSet& maps, int grid, cudaStream_t st);
int count_tc_smem_bytes(int I, int wseg, int ot_max, int wrows, int direct);
int count_tc_tile();
int launch_cand_params(const ProbDev* dprob, int first_region, int n_patch, int per_region, const bsh_cand* cands,
                       const int32_t* n_cands, int stat, const bsh_post_params* pp, double* params, double* sig,
                       int32_t* valid, cudaStream_t st);
void launch_tables(const ProbDev& hp, const ProbDev* dprob, int mode, unsigned* status, cudaStream_t st);
void launch_peakgram(const float* power, int N, int K, int window, double rho_th, float* rho,
                     uint32_t* bits, int W, cudaStream_t st);
int launch_weights(const double* sky, int S, const double* arms, const double* Sn, int N, int norm,
                   int dtype, void* w, double* sum_w, double* sum_w2, unsigned* status, cudaStream_t st);

struct MergeArgs {
    const ProbDev* probs;
    int n_probs;
    const int32_t* region_problem;   // [regions]
    const int32_t* region_visit_off; // [regions + 1]
    const int32_t* region_visits;    // [sum visits]
    const Entry* visit_buf;
    const int32_t* visit_count;
    int cap, top_k;
    Entry* scratch;                  // [regions][top_k]
    bsh_cand* out;
    int32_t* n_out;
    unsigned* status;
};
void launch_merge(const MergeArgs& a, int regions, cudaStream_t st);

struct PowerArgs {
    const ProbDev* probs;
    int n_probs;
    const int32_t* region_problem;
    bsh_cand* cands;
    const int32_t* n_cands;
    int top_k, n_cf;
    bsh_cand* final_list;
    int32_t* n_final;
    unsigned* status;
};
void launch_power(const PowerArgs& a, int regions, cudaStream_t st);
void launch_precision(const ProbDev* dprob, int s_begin, int s_end, unsigned long long* counts, cudaStream_t st);
void launch_bins(const ProbDev* dprob, const int64_t* ids, int n, int32_t* bins, unsigned* status, cudaStream_t st);

}  // namespace bsh
