// C ABI of libbsh: argument validation, fixed-point scale selection, the
// static persistent schedule, workspace layout, launches, status, graphs.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "bsh_internal.cuh"

namespace bsh {
int count_smem_bytes(int mode, int I, int wseg, int ot_max, int wrows, int threads, int acc, int direct);
int count_c_stride(int I);
}

using namespace bsh;

namespace {

__device__ unsigned g_status_word;

constexpr int kVersion = 10000;

int cuda_fail(cudaError_t e) { return e == cudaSuccess ? BSH_OK : BSH_ERR_CUDA; }

// Device address of the status word for the current device (looked up once per device).
unsigned* status_ptr() {
    static std::mutex mu;
    static unsigned* ptrs[64] = {nullptr};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(mu);
    if (!ptrs[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_status_word) != cudaSuccess) return nullptr;
        ptrs[dev] = static_cast<unsigned*>(p);
    }
    return ptrs[dev];
}

int ceil_log2(double x) {
    int e = 0;
    double p = 1.0;
    if (x <= 1.0) {
        while (p / 2.0 >= x && e > -200) { p /= 2.0; --e; }
        return e;
    }
    while (p < x && e < 200) { p *= 2.0; ++e; }
    return e;
}

bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

// Fixed-point scales for the track of one problem (see bsh_internal.cuh).
// Om_max bounds |c| = |Omega g| over every orbit row (Omega (1 + |kappa| + |eta|)).
int choose_fixed_point(double F_max, double v_max, double ap_max, double Om_max, double phi, FixedPoint* fp) {
    const double ymax = F_max * (v_max + ap_max * Om_max) + 2.0;
    fp->s_vn = 30 - ceil_log2(v_max * (1.0 + 1e-9));
    fp->s_c = 30 - ceil_log2(Om_max * (1.0 + 1e-9));
    fp->s_a = 30 - ceil_log2(std::max(ap_max, 1.0 / 1048576.0) * (1.0 + 1e-12));
    const double C_max = F_max * Om_max * (1.0 + 1e-9);
    const int sC_cap = 30 - ceil_log2(C_max);
    fp->s_y = std::min(30 - ceil_log2(ymax), fp->s_a + sC_cap - 32);
    fp->s_C = fp->s_y + 32 - fp->s_a;
    fp->sh_v = fp->s_vn + 1 - fp->s_y;
    fp->sh_c = fp->s_c + 1 - fp->s_C;
    if (fp->s_y < 18 || fp->sh_v < 0 || fp->sh_c < 0 || fp->sh_v > 62 || fp->sh_c > 62) return BSH_ERR_RANGE;
    fp->off_q = (int)std::llround((phi + 0.5) * std::ldexp(1.0, fp->s_y));
    // error bound of v in units of 2^-s_y (see bsh_internal.cuh)
    const double u = std::ldexp(1.0, fp->s_y);
    const double eZ = 0.5 + F_max * std::ldexp(1.0, -fp->s_vn - 1) * u;
    const double eC = 0.5 + F_max * std::ldexp(1.0, -fp->s_c - 1) * std::ldexp(1.0, fp->s_C);
    const double ea = 0.5;
    const double prod = (ap_max * std::ldexp(1.0, fp->s_a) * eC + C_max * std::ldexp(1.0, fp->s_C) * ea + ea * eC) /
                        4294967296.0;
    const double cosulp = F_max * Om_max * ap_max * 4.0e-16 * u;   // libm-level differences of cos / sin
    fp->eps = eZ + 1.0 + prod + cosulp + 1.0;
    fp->M = (int)std::ceil(2.0 * fp->eps) + 4;
    if (fp->M * 8 > (1 << fp->s_y)) return BSH_ERR_RANGE;
    // slope margin of the reference-template test: |v(j) - v(j0 + 15)| <= 16 |D| 2^s_y for the
    // block's templates, |D| <= |vn| + a_p |c|, |vn| <= (|vn_q| + 1) 2^-s_vn, |c| <= Om_max
    // (a margin of a whole cell or more only sends every block to the two-ended test)
    const double binpart = 16.0 * ap_max * Om_max * (1.0 + 1e-9) * u;
    fp->mg_a = (int)std::min(std::ceil(binpart) + fp->M + 2, u);
    if (fp->s_vn - fp->s_y - 4 < 0) return BSH_ERR_RANGE;
    fp->mg_k = std::min(30, fp->s_vn - fp->s_y - 4);   // a smaller shift only rounds the margin up
    return BSH_OK;
}

struct ProbHost {
    bsh_problem d;                         // caller descriptor (device pointers)
    std::vector<double> orb;               // [nOT][4] Omega, t_asc, kappa, eta
    std::vector<int32_t> brow;             // [B] orbit row of each binary template
    std::vector<double> bap;               // [B] a_p of each binary template
    std::vector<int32_t> bapq;             // [B] fixed-point a_p (set with the scales)
    std::vector<int64_t> ps;
    std::vector<int32_t> patch_of_s;
    ProbDev pd;                            // filled at create (sizes) and bind (pointers)
    size_t off_orb, off_brow, off_bap, off_bapq, off_ps, off_pos, off_vnq, off_cq, off_c64, off_w;
};

bool uses_bank(const bsh_problem& d) { return d.n_orbit > 0; }

// Binary templates of a problem as orbit rows plus (row, a_p) per template: the explicit bank
// as given, or the grid written out in its template order
// b = (((iOm * n_T + iT) * n_kap + ik) * n_eta + ie) * n_ap + iap.
void expand_binaries(ProbHost& h, const bsh_problem& d) {
    h.orb.clear();
    h.brow.clear();
    h.bap.clear();
    if (uses_bank(d)) {
        h.orb.assign(d.orbit, d.orbit + 4 * (size_t)d.n_orbit);
        h.brow.assign(d.bank_orbit, d.bank_orbit + d.n_bank);
        h.bap.assign(d.bank_ap, d.bank_ap + d.n_bank);
        return;
    }
    const int nk = std::max(1, d.n_kappa), ne = std::max(1, d.n_eta);
    for (int iOm = 0; iOm < d.n_Om; ++iOm)
        for (int iT = 0; iT < d.n_T; ++iT)
            for (int ik = 0; ik < nk; ++ik)
                for (int ie = 0; ie < ne; ++ie) {
                    h.orb.push_back(d.Omega[iOm]);
                    h.orb.push_back(d.T_asc[(size_t)iOm * d.n_T + iT]);
                    h.orb.push_back(d.n_kappa > 0 ? d.kappa[ik] : 0.0);
                    h.orb.push_back(d.n_eta > 0 ? d.eta[ie] : 0.0);
                }
    const int rows = (int)(h.orb.size() / 4);
    h.brow.reserve((size_t)rows * d.n_ap);
    h.bap.reserve((size_t)rows * d.n_ap);
    for (int r = 0; r < rows; ++r)
        for (int k = 0; k < d.n_ap; ++k) {
            h.brow.push_back(r);
            h.bap.push_back(d.a_p[k]);
        }
}

// Binary templates of a problem (grid size or bank size).
long long binary_count(const bsh_problem& d) {
    if (uses_bank(d)) return d.n_bank;
    return (long long)d.n_ap * d.n_Om * d.n_T * std::max(1, d.n_kappa) * std::max(1, d.n_eta);
}

// Largest a_p and bound on |Omega g| = |c| over the orbit rows (g of Eq. (14)).
void binary_bounds(const ProbHost& h, double* ap_max, double* c_max) {
    double a = 0.0, c = 0.0;
    for (double x : h.bap) a = std::max(a, x);
    for (size_t r = 0; r < h.orb.size() / 4; ++r)
        c = std::max(c, h.orb[4 * r] * (1.0 + std::fabs(h.orb[4 * r + 2]) + std::fabs(h.orb[4 * r + 3])));
    *ap_max = a;
    *c_max = c;
}

}  // namespace

constexpr int kDefaultWaitPolls = 1 << 22;   // about a second or more of polling

struct bsh_plan {
    int n = 0;
    std::vector<ProbHost> P;
    bsh_count_options opt{};
    int mode = BSH_MODE_BATCHED;           // BSH_MODE_LUT plans run as BATCHED with lut = 1
    int lut = 0;
    int threads = 256, chunk = 128, ctas = 0, num_sms = 152;
    int wseg_max = 4, ot_max = 1, wrows = 1, smem = 0, cap = 0, top_k = 1000;
    int regions = 0, visits = 0, visit_cap = 0;
    size_t ws_cap = 0;                     // workspace bytes: the largest of the tuning candidates
    double tuned_rate = 0.0;
    int acc_mode = 0;                      // weighted accumulation variant (autotuned); 2 = tensor cores
    int direct_opt = -1;                   // per-term C values: -1 automatic, 0 off, 1 on
    int direct = 0;                        // the choice in effect
    int direct_tuned = -1;                 // the autotuner's choice under direct_opt = -1 (-1: none yet)
    int one_cta = 0;                       // 1: one CTA per SM with the unshrunk stage (autotuned)
    int wait_polls = kDefaultWaitPolls;    // staging-barrier polls before a wait gives up
    int skip_stage = -1;                   // test hook: stage left unissued in every CTA (-1: none)
    std::vector<int64_t> cta_item;
    std::vector<int32_t> cta_visit;
    int pools = 0;                    // batched: CTAs c + m * pools share pool c
    int pool_size = 0;                // CTAs per pool
    std::vector<int64_t> pool_item;   // [pools + 1] item range of each pool
    std::vector<int32_t> pool_sweep;  // [2 * pools] walk rotation r and sweep length P
    std::vector<int32_t> pool_run;    // [pools + 1] runs of each pool in run_step
    std::vector<int64_t> run_step;    // [runs] first walk step of each run
    std::vector<int32_t> region_problem, region_visit_off, region_visits;
    // plain mode: per-region schedules
    std::vector<int32_t> pl_off, pl_ctas;
    // workspace layout
    size_t off_probs = 0, off_cta_item = 0, off_cta_visit = 0, off_pool_item = 0, off_pool_sweep = 0,
           off_pool_run = 0, off_run_step = 0, off_pool_next = 0, off_vbuf = 0, off_vcount = 0;
    size_t off_rprob = 0, off_rvoff = 0, off_rvis = 0, off_scratch = 0, off_dense = 0, ws_size = 0;
    unsigned char* ws = nullptr;
    bool bound = false;
    TmapSet maps{};
    // graph
    cudaGraphExec_t gexec = nullptr;
    cudaGraph_t graph = nullptr;
    cudaStream_t cap_stream = nullptr;
    const void* g_args[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    int g_ncf = 0;
};

namespace {

size_t al(size_t x) { return (x + 255) & ~size_t(255); }

// Binary templates per work item: the CTA size, or the tensor-core kernel's fixed tile.
int tile_b(const bsh_plan* p) { return p->acc_mode == 2 ? count_tc_tile() : p->threads; }

// Whether the tensor-core accumulation applies: the exact-track batched count with 256-thread CTAs.
bool tc_ok(const bsh_plan* p) { return p->mode == BSH_MODE_BATCHED && !p->lut && p->threads == 256; }

// Tile shapes the autotuner considers (the first is the default).
std::vector<int> tune_threads(const bsh_plan* p) {
    if (p->opt.threads) return {p->opt.threads};
    if (p->mode == BSH_MODE_PLAIN) return {256};
    return {256, 128};
}
std::vector<int> tune_chunks(const bsh_plan* p) {
    if (p->opt.sft_chunk) return {p->opt.sft_chunk};
    if (p->mode == BSH_MODE_PLAIN) return {128};
    return {128, 64, 256};
}

int build_schedule(bsh_plan* p, long long item_limit = -1);

// f0 block and binary tile of item `loc` of a problem, in the kernels' item order: sky
// points in turn, inside a sky point binary tiles, then f0 blocks.
void item_fb_bt(const ProbHost& h, long long loc, int* fb, int* bt) {
    const ProbDev& pd = h.pd;
    const long long per_s = (long long)pd.n_fb * pd.n_bt;
    const int rem = (int)(loc % per_s);
    *bt = rem / pd.n_fb;
    *fb = rem % pd.n_fb;
}

// The contiguous item runs, in walk order, of a pool with range [a, a + len), sweep length P
// and rotation r (the batched kernels' walk): sweep j starts at offset r of
// [a + jP, a + (j+1)P) and wraps round; a last partial sweep of m <= r items (inside one sky
// point, whose tiles P - r ... P - r + m - 1 it holds) starts at its tile that is a multiple
// of m.
template <class F>
void walk_runs(long long a, long long len, long long P, long long r, F&& run) {
    if (len <= 0) return;
    if (r == 0) {
        run(a, a + len);
        return;
    }
    for (long long j0 = 0; j0 < len; j0 += P) {
        const long long m = std::min(P, len - j0);
        const long long e = std::max(m - r, 0LL);
        if (e == 0 && m < P) {
            const long long rho = (m - (P - r) % m) % m;
            run(a + j0 + rho, a + j0 + m);
            if (rho > 0) run(a + j0, a + j0 + rho);
            continue;
        }
        if (e > 0) run(a + j0 + r, a + j0 + r + e);
        if (m - e > 0) run(a + j0, a + j0 + (m - e));
    }
}
int upload_plan(bsh_plan* p, cudaStream_t st);

int validate_problem(const bsh_problem& d) {
    if (d.N <= 0 || d.K <= 0 || d.W < (d.K + 31) / 32 || d.W % 4 != 0) return BSH_ERR_ARG;
    if (!d.bits || !d.w || !d.sum_w || !d.sum_w2 || !d.v || !d.t || !d.sky) return BSH_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(d.bits) % 16 != 0) return BSH_ERR_ARG;
    if (d.w_dtype < BSH_F64 || d.w_dtype > BSH_BF16) return BSH_ERR_ARG;
    if (d.n_f0 <= 0 || d.S <= 0 || d.n_patch <= 0 || !d.patch_start) return BSH_ERR_ARG;
    if (uses_bank(d)) {
        if (d.n_bank <= 0 || !d.orbit || !d.bank_orbit || !d.bank_ap) return BSH_ERR_ARG;
        if (d.n_bank > (1 << 30)) return BSH_ERR_RANGE;
        for (int r = 0; r < d.n_orbit; ++r) {
            const double* o = d.orbit + 4 * (size_t)r;
            if (!finite_pos(o[0]) || !std::isfinite(o[1]) || !(std::fabs(o[2]) <= 0.5) || !(std::fabs(o[3]) <= 0.5))
                return BSH_ERR_ARG;
        }
        for (int b = 0; b < d.n_bank; ++b) {
            if (d.bank_orbit[b] < 0 || d.bank_orbit[b] >= d.n_orbit) return BSH_ERR_ARG;
            if (b > 0 && d.bank_orbit[b] < d.bank_orbit[b - 1]) return BSH_ERR_ARG;
            if (!(d.bank_ap[b] >= 0.0) || !std::isfinite(d.bank_ap[b])) return BSH_ERR_ARG;
        }
    } else if (d.n_ap <= 0 || d.n_Om <= 0 || d.n_T <= 0 || !d.a_p || !d.Omega || !d.T_asc) {
        return BSH_ERR_ARG;
    }
    if (!finite_pos(d.v_max) || !std::isfinite(d.F0) || d.F0 <= 0.0) return BSH_ERR_ARG;
    const double F2 = 2.0 * d.F0;
    if (F2 != std::floor(F2) || F2 + 2.0 * (d.n_f0 + 64) > 2147483000.0) return BSH_ERR_ARG;
    if (!(d.rho_th > 0.0) || !std::isfinite(d.rho_th)) return BSH_ERR_ARG;
    if (d.patch_start[0] != 0 || d.patch_start[d.n_patch] != d.S) return BSH_ERR_ARG;
    for (int p = 0; p < d.n_patch; ++p)
        if (d.patch_start[p + 1] < d.patch_start[p]) return BSH_ERR_ARG;
    if (uses_bank(d)) return BSH_OK;
    for (int k = 0; k < d.n_ap; ++k)
        if (!(d.a_p[k] >= 0.0) || !std::isfinite(d.a_p[k])) return BSH_ERR_ARG;
    for (int k = 0; k < d.n_Om; ++k)
        if (!finite_pos(d.Omega[k])) return BSH_ERR_ARG;
    for (int k = 0; k < d.n_Om * d.n_T; ++k)
        if (!std::isfinite(d.T_asc[k])) return BSH_ERR_ARG;
    if (d.n_kappa < 0 || d.n_eta < 0 || (d.n_kappa > 0 && !d.kappa) || (d.n_eta > 0 && !d.eta))
        return BSH_ERR_ARG;
    for (int k = 0; k < d.n_kappa; ++k)
        if (!(std::fabs(d.kappa[k]) <= 0.5)) return BSH_ERR_ARG;
    for (int k = 0; k < d.n_eta; ++k)
        if (!(std::fabs(d.eta[k]) <= 0.5)) return BSH_ERR_ARG;
    if (binary_count(d) > (1LL << 30)) return BSH_ERR_RANGE;
    return BSH_OK;
}

int prepare_problem(bsh_plan* p, ProbHost& h) {
    const bsh_problem& d = h.d;
    ProbDev& pd = h.pd;
    std::memset(&pd, 0, sizeof(pd));
    pd.N = d.N;
    pd.K = d.K;
    pd.W = d.W;
    pd.k_lo = d.k_lo;
    pd.n_f0 = d.n_f0;
    pd.S = d.S;
    const long long rows = (long long)(h.orb.size() / 4);
    const long long B = (long long)h.bap.size();
    if (B > (1LL << 30) || B <= 0) return BSH_ERR_RANGE;
    pd.nOT = (int)rows;
    pd.B = (int)B;
    pd.n_patch = d.n_patch;
    pd.w_dtype = d.w_dtype;
    pd.F0 = d.F0;
    pd.G0 = (int)std::floor(d.F0);
    const int nb = (d.n_f0 + JW - 1) / JW;
    pd.JB = (d.n_f0 + nb - 1) / nb;
    pd.n_fb = (d.n_f0 + pd.JB - 1) / pd.JB;
    pd.n_bt = (pd.B + tile_b(p) - 1) / tile_b(p);
    pd.p_th = std::exp(-d.rho_th);
    pd.v_max = d.v_max;
    // patch template counts must fit a 32-bit local id
    for (int q = 0; q < d.n_patch; ++q) {
        const double nt = (double)(h.ps[q + 1] - h.ps[q]) * (double)B * d.n_f0;
        if (nt >= 4294967295.0) return BSH_ERR_RANGE;
    }
    double ap_max = 0.0, Om_max = 0.0;
    binary_bounds(h, &ap_max, &Om_max);
    const int j_last = (pd.n_fb - 1) * pd.JB + JW;             // last f0 offset evaluated (+1 for a crossing)
    const double F_eval = d.F0 + j_last;
    const double phi = d.F0 - std::floor(d.F0);
    int rc = choose_fixed_point(F_eval, d.v_max, ap_max, Om_max, phi, &pd.fp);
    if (rc) return rc;
    const double ymax = F_eval * (d.v_max + ap_max * Om_max);
    pd.o_max = (int)std::ceil(ymax) + 2;
    pd.o_min = -pd.o_max;
    // band check: every valid template stays inside [k_lo, k_lo + K)
    const double Fv_max = d.F0 + d.n_f0 - 1;
    const double yv = Fv_max * (d.v_max + ap_max * Om_max);
    const long long kmin = (long long)std::floor(d.F0 - yv + 0.5) - 1;
    const long long kmax = (long long)std::floor(Fv_max + yv + 0.5) + 1;
    if (kmin < d.k_lo || kmax >= (long long)d.k_lo + d.K) return BSH_ERR_RANGE;
    // staged segment width
    int wseg = 4;
    for (int fb = 0; fb < pd.n_fb; ++fb) {
        const int Gj0 = pd.G0 + fb * pd.JB;
        int lo_bin = Gj0 + pd.o_min - 1 - d.k_lo;
        lo_bin = std::max(lo_bin, 0);
        const int c0 = (lo_bin >> 5) & ~3;
        const int hi_bin = Gj0 + 31 + pd.o_max + 1 - d.k_lo;
        const int w = ((hi_bin >> 5) - c0 + 2 + 3) & ~3;
        wseg = std::max(wseg, w);
    }
    if (wseg > 64) return BSH_ERR_RANGE;
    pd.Wseg = wseg;
    // a_p in fixed point
    h.bapq.resize(h.bap.size());
    for (size_t k = 0; k < h.bap.size(); ++k) h.bapq[k] = (int32_t)std::llround(std::ldexp(h.bap[k], pd.fp.s_a));
    // patch of each sky point
    h.patch_of_s.assign(d.S, 0);
    for (int q = 0; q < d.n_patch; ++q)
        for (int64_t s = h.ps[q]; s < h.ps[q + 1]; ++s) h.patch_of_s[s] = q;
    return BSH_OK;
}

}  // namespace

extern "C" {

const char* bsh_error_string(int status) {
    switch (status) {
        case BSH_OK: return "ok";
        case BSH_ERR_ARG: return "invalid argument";
        case BSH_ERR_RANGE: return "track outside the loaded band or parameter outside the fixed-point range";
        case BSH_ERR_TIMEOUT: return "bounded device wait expired";
        case BSH_ERR_CUDA: return "CUDA runtime error";
        case BSH_ERR_WORKSPACE: return "workspace missing or too small";
        case BSH_ERR_STATE: return "call order violated";
        default: return "unknown status";
    }
}

int bsh_version(void) { return kVersion; }

int bsh_sync_status(bsh_stream stream) {
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return BSH_ERR_CUDA;
    unsigned* sp = status_ptr();
    if (!sp) return BSH_ERR_CUDA;
    unsigned v = 0;
    if (cudaMemcpy(&v, sp, sizeof(v), cudaMemcpyDeviceToHost) != cudaSuccess) return BSH_ERR_CUDA;
    const unsigned zero = 0;
    if (cudaMemcpy(sp, &zero, sizeof(zero), cudaMemcpyHostToDevice) != cudaSuccess) return BSH_ERR_CUDA;
    if (v & ST_TIMEOUT) return BSH_ERR_TIMEOUT;
    if (v & ST_RANGE) return BSH_ERR_RANGE;
    if (v & ST_ARG) return BSH_ERR_ARG;
    return BSH_OK;
}

int bsh_make_peakgram(const float* power, int N, int K, int median_window, double rho_th, float* rho_out,
                      uint32_t* bits, int W, bsh_stream stream) {
    if (N < 0 || K <= 0 || W < (K + 31) / 32 || !bits || (N > 0 && !power)) return BSH_ERR_ARG;
    if (median_window < 0 || (median_window > 0 && (median_window % 2 == 0 || median_window > K)))
        return BSH_ERR_ARG;
    if (median_window > 0 && ((size_t)K + (size_t)W) * sizeof(float) > 200 * 1024) return BSH_ERR_ARG;
    if (!std::isfinite(rho_th)) return BSH_ERR_ARG;
    launch_peakgram(power, N, K, median_window, rho_th, rho_out, bits, W, (cudaStream_t)stream);
    return cuda_fail(cudaGetLastError());
}

int bsh_weights(const double* sky, int S, const double* arms, const double* Sn, int N, int normalize, int dtype,
                void* w, double* sum_w, double* sum_w2, bsh_stream stream) {
    if (S < 0 || N <= 0 || !arms || !Sn || (S > 0 && (!sky || !w))) return BSH_ERR_ARG;
    if (dtype < BSH_F64 || dtype > BSH_BF16 || (normalize != 0 && normalize != 1)) return BSH_ERR_ARG;
    unsigned* sp = status_ptr();
    if (!sp) return BSH_ERR_CUDA;
    launch_weights(sky, S, arms, Sn, N, normalize, dtype, w, sum_w, sum_w2, sp, (cudaStream_t)stream);
    return cuda_fail(cudaGetLastError());
}

int bsh_plan_create(const bsh_problem* problems, int n_problems, const bsh_count_options* opt, bsh_plan** out) {
    if (!out) return BSH_ERR_ARG;
    *out = nullptr;
    if (!problems || n_problems < 1 || n_problems > MAX_PROBLEMS || !opt) return BSH_ERR_ARG;
    if (opt->mode != BSH_MODE_BATCHED && opt->mode != BSH_MODE_PLAIN && opt->mode != BSH_MODE_LUT)
        return BSH_ERR_ARG;
    if (opt->top_k < 1 || opt->top_k > 16384) return BSH_ERR_ARG;
    if (opt->threads != 0 && opt->threads != 128 && opt->threads != 256) return BSH_ERR_ARG;
    if (opt->sft_chunk != 0 && opt->sft_chunk != 64 && opt->sft_chunk != 128 && opt->sft_chunk != 256)
        return BSH_ERR_ARG;
    if (opt->ctas_per_sm < 0 || opt->ctas_per_sm > 8) return BSH_ERR_ARG;
    for (int q = 0; q < n_problems; ++q) {
        const int rc = validate_problem(problems[q]);
        if (rc) return rc;
    }
    bsh_plan* p = new bsh_plan();
    p->n = n_problems;
    p->opt = *opt;
    p->mode = opt->mode == BSH_MODE_LUT ? BSH_MODE_BATCHED : opt->mode;
    p->lut = opt->mode == BSH_MODE_LUT ? 1 : 0;
    p->top_k = opt->top_k;
    p->threads = opt->threads ? opt->threads : 256;
    p->chunk = opt->sft_chunk ? opt->sft_chunk : 128;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && nsm > 0)
        p->num_sms = nsm;
    else
        cudaGetLastError();
    p->P.resize(n_problems);
    for (int q = 0; q < n_problems; ++q) {
        ProbHost& h = p->P[q];
        h.d = problems[q];
        const bsh_problem& d = problems[q];
        expand_binaries(h, d);
        h.ps.assign(d.patch_start, d.patch_start + d.n_patch + 1);
        h.d.a_p = nullptr;
        h.d.Omega = nullptr;
        h.d.T_asc = nullptr;
        h.d.kappa = nullptr;
        h.d.eta = nullptr;
        h.d.orbit = nullptr;
        h.d.bank_orbit = nullptr;
        h.d.bank_ap = nullptr;
        h.d.patch_start = nullptr;
    }
    // size the workspace for every tile shape the autotuner may pick
    size_t cap = 0;
    int first_rc = -1;
    for (int t : tune_threads(p))
        for (int c : tune_chunks(p))
            for (int v = 0; v < 12; ++v) {
                p->threads = t;
                p->chunk = c;
                p->acc_mode = v % 3;
                p->one_cta = (v / 3) & 1;
                p->direct_tuned = v / 6;
                const int rc = build_schedule(p);
                if (first_rc < 0) first_rc = rc;
                if (rc == BSH_OK) cap = std::max(cap, p->ws_size);
            }
    p->threads = tune_threads(p)[0];
    p->chunk = tune_chunks(p)[0];
    p->acc_mode = 0;
    p->one_cta = 0;
    p->direct_tuned = -1;
    const int rc = build_schedule(p);
    if (rc) {
        delete p;
        return rc;
    }
    p->ws_cap = std::max(cap, p->ws_size);
    *out = p;
    return BSH_OK;
}

void bsh_plan_destroy(bsh_plan* p) {
    if (!p) return;
    if (p->gexec) cudaGraphExecDestroy(p->gexec);
    if (p->graph) cudaGraphDestroy(p->graph);
    if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
    delete p;
}

size_t bsh_plan_workspace_size(const bsh_plan* p) { return p ? p->ws_cap : 0; }

int bsh_debug_pool_walk(const bsh_plan* p, int pool, int64_t* items, int64_t cap, int64_t* n_items, int* n_pools,
                        int* pool_size) {
    if (!p) return BSH_ERR_ARG;
    if (p->mode != BSH_MODE_BATCHED) return BSH_ERR_STATE;
    if (n_pools) *n_pools = p->pools;
    if (pool_size) *pool_size = p->pool_size;
    if (pool < 0 || pool >= p->pools) return BSH_ERR_ARG;
    const long long a = p->pool_item[pool], len = p->pool_item[pool + 1] - a;
    if (n_items) *n_items = len;
    if (!items) return BSH_OK;
    if (cap < len) return BSH_ERR_ARG;
    long long k = 0;
    walk_runs(a, len, p->pool_sweep[2 * pool + 1], p->pool_sweep[2 * pool], [&](long long x, long long y) {
        for (long long i = x; i < y; ++i) items[k++] = i;
    });
    return BSH_OK;
}
int bsh_plan_num_regions(const bsh_plan* p) { return p ? p->regions : 0; }
int bsh_plan_first_region(const bsh_plan* p, int q) {
    if (!p || q < 0 || q >= p->n) return -1;
    return p->P[q].pd.region_base;
}

}  // extern "C"

namespace {

int build_schedule(bsh_plan* p, long long item_limit) {
    if (p->acc_mode == 2 && !tc_ok(p)) p->acc_mode = 0;
    // tile shapes
    p->ot_max = 1;
    p->wrows = 1;
    // orbit rows spanned by one binary tile (CTA) and by one warp's 32 templates
    for (auto& h : p->P) {
        const int B = (int)h.brow.size();
        for (int b0 = 0; b0 < B; b0 += tile_b(p)) {
            const int b1 = std::min(b0 + tile_b(p), B) - 1;
            p->ot_max = std::max(p->ot_max, h.brow[b1] - h.brow[b0] + 1);
            for (int w0 = b0; w0 <= b1; w0 += 32) {
                const int w1 = std::min(w0 + 31, B - 1);
                p->wrows = std::max(p->wrows, h.brow[w1] - h.brow[w0] + 1);
            }
        }
    }
    // orbit rows shared by few templates (banks): form C per term rather than per warp
    const bool auto_direct = p->direct_tuned >= 0 ? p->direct_tuned == 1 : p->wrows > 4;
    p->direct = p->mode == BSH_MODE_BATCHED && (p->direct_opt == 1 || (p->direct_opt < 0 && auto_direct)) ? 1 : 0;
    // the per-term variant accumulates by predicated adds or on the tensor cores
    if (p->direct && p->acc_mode == 1) p->acc_mode = 0;
    int region = 0;
    long long items = 0;
    for (auto& h : p->P) {
        const int rc = prepare_problem(p, h);
        if (rc) return rc;
        h.pd.region_base = region;
        region += h.d.n_patch;
        p->wseg_max = std::max(p->wseg_max, h.pd.Wseg);
    }
    p->regions = region;
    // chunk size: shrink until the CTAs that the register budget allows per SM
    // (512 threads) also fit its shared memory; else (or when one CTA per SM is
    // asked for) settle for one CTA per SM
    const int blocks_target = p->opt.ctas_per_sm > 1 ? p->opt.ctas_per_sm : 512 / p->threads;
    const int smem_two = (227 * 1024) / blocks_target - 1024, smem_one = 220 * 1024;
    const int chunk0 = p->chunk;
    const bool one = p->one_cta || p->opt.ctas_per_sm == 1;
    bool fits_two = false;
    while (!one) {
        p->smem = p->acc_mode == 2 ? count_tc_smem_bytes(p->chunk, p->wseg_max, p->ot_max, p->wrows, p->direct)
                                   : count_smem_bytes(p->mode, p->chunk, p->wseg_max, p->ot_max, p->wrows, p->threads,
                                                      p->acc_mode, p->direct);
        fits_two = p->smem <= smem_two;
        if (fits_two || p->chunk <= 32) break;
        p->chunk /= 2;
    }
    if (!fits_two) {
        p->chunk = chunk0;
        while (true) {
            p->smem = p->acc_mode == 2 ? count_tc_smem_bytes(p->chunk, p->wseg_max, p->ot_max, p->wrows, p->direct)
                                       : count_smem_bytes(p->mode, p->chunk, p->wseg_max, p->ot_max, p->wrows,
                                                          p->threads, p->acc_mode, p->direct);
            if (p->smem <= smem_one || p->chunk <= 32) break;
            p->chunk /= 2;
        }
    }
    if (p->smem > smem_one) return BSH_ERR_RANGE;
    std::vector<long long> cum_cost(p->n + 1, 0);
    for (int q = 0; q < p->n; ++q) {
        ProbDev& pd = p->P[q].pd;
        pd.Np = (pd.N + 255) / 256 * 256;
        pd.item_begin = items;
        pd.n_items = (long long)pd.S * pd.n_fb * pd.n_bt;
        pd.cost = (pd.N + p->chunk - 1) / p->chunk + 1;
        items += pd.n_items;
        cum_cost[q + 1] = cum_cost[q] + pd.n_items * pd.cost;
    }
    const long long all_items = items;
    const long long total_items = item_limit >= 0 ? std::min(item_limit, all_items) : all_items;
    const int cps = p->opt.ctas_per_sm ? p->opt.ctas_per_sm
                    : (p->mode == BSH_MODE_BATCHED && fits_two ? blocks_target : 1);
    const int k = p->top_k;
    // region item ranges
    std::vector<long long> r_begin(p->regions + 1, 0);
    std::vector<int> r_prob(p->regions);
    for (int q = 0; q < p->n; ++q) {
        const ProbDev& pd = p->P[q].pd;
        const long long per_s = (long long)pd.n_fb * pd.n_bt;
        for (int pt = 0; pt < pd.n_patch; ++pt) {
            r_begin[pd.region_base + pt] = pd.item_begin + p->P[q].ps[pt] * per_s;
            r_prob[pd.region_base + pt] = q;
        }
    }
    r_begin[p->regions] = all_items;
    p->region_problem.assign(r_prob.begin(), r_prob.end());
    std::vector<std::vector<int32_t>> rvis(p->regions);
    if (p->mode == BSH_MODE_BATCHED) {
        long long C = (long long)p->num_sms * cps;
        C = std::max(1LL, std::min(C, total_items));
        p->ctas = (int)C;
        p->cta_item.assign(C + 1, 0);
        const long long T = cum_cost[p->n];
        for (long long c = 0; c <= C; ++c) {
            long long it;
            if (total_items < all_items) {
                it = total_items * c / C;     // a slice for the autotuner: even split
            } else {
                const long long X = (long long)((__int128)T * c / C);
                int q = 0;
                while (q + 1 < p->n && X >= cum_cost[q + 1]) ++q;
                it = p->P[q].pd.item_begin + (X - cum_cost[q]) / p->P[q].pd.cost;
            }
            if (c == C) it = total_items;
            p->cta_item[c] = std::min(it, total_items);
        }
        for (long long c = 1; c <= C; ++c) p->cta_item[c] = std::max(p->cta_item[c], p->cta_item[c - 1]);
        p->cta_visit.assign(C + 1, 0);   // (the plain kernel's)
        // pools: CTAs q + m H (m < G) share pool q, the cost-balanced range of as many
        // consecutive CTA slots as it has CTAs.  Pools of four balance best, but a pool's range
        // then spans twice the binary tiles of a pair's and the pools drift further apart in
        // tiles; a fixed-point orbit table larger than half the L2 pays for that in DRAM
        // re-reads (3.5x the bytes on the metric bank), so such plans use pairs.
        size_t table = 0;
        for (const auto& h : p->P) table = std::max(table, (size_t)h.pd.nOT * (size_t)h.pd.Np * sizeof(int32_t));
        const int G = table > ((size_t)64 << 20) ? 2 : kPoolMax;
        p->pool_size = G;
        const long long H = (C + G - 1) / G;
        p->pools = (int)H;
        auto members = [&](long long q) {
            int n = 0;
            for (int m = 0; m < G; ++m) n += q + m * H < C ? 1 : 0;
            return n;
        };
        p->pool_item.assign(H + 1, 0);
        for (long long q = 0, slot = 0; q < H; slot += members(q), ++q) p->pool_item[q] = p->cta_item[slot];
        p->pool_item[H] = p->cta_item[C];
        // the walk of each pool: a range inside one problem, with at most one region boundary
        // inside, sweeps that problem's sky points from the first binary tile of its first whole
        // sky point (see walk_runs); any other range is walked in order
        p->pool_sweep.assign(2 * H, 0);
        for (long long q = 0; q < H; ++q) {
            const long long a = p->pool_item[q], b = p->pool_item[q + 1];
            if (a >= b) continue;
            int pi = 0;
            while (pi + 1 < p->n && a >= p->P[pi + 1].pd.item_begin) ++pi;
            const ProbDev& pd = p->P[pi].pd;
            const long long P = (long long)pd.n_fb * pd.n_bt;
            if (b > pd.item_begin + pd.n_items || P <= 0) continue;   // spans problems
            const long long r = (P - (a - pd.item_begin) % P) % P;
            if (r >= b - a) continue;                                  // no sky point boundary inside
            int inner = 0;
            long long prev = a;
            for (auto it = std::upper_bound(r_begin.begin(), r_begin.end(), a); it != r_begin.end() && *it < b; ++it)
                if (*it != prev) {
                    ++inner;
                    prev = *it;
                }
            if (inner > 1) continue;
            p->pool_sweep[2 * q] = (int32_t)r;
            p->pool_sweep[2 * q + 1] = (int32_t)P;
        }
        // runs: the maximal stretches of one region along each pool's walk; run j owns visits
        // G j + m, one for each CTA m of the pool
        p->pool_run.assign(H + 1, 0);
        p->run_step.clear();
        for (long long q = 0; q < H; ++q) {
            p->pool_run[q] = (int32_t)p->run_step.size();
            const int nm = members(q);
            int last = -1;
            long long steps = 0;   // walk steps before the current stretch
            walk_runs(p->pool_item[q], p->pool_item[q + 1] - p->pool_item[q], p->pool_sweep[2 * q + 1],
                      p->pool_sweep[2 * q], [&](long long a, long long b) {
                          int r = (int)(std::upper_bound(r_begin.begin(), r_begin.end(), a) - r_begin.begin()) - 1;
                          while (r < p->regions && r_begin[r] < b) {
                              if (r_begin[r + 1] > r_begin[r] && r_begin[r + 1] > a && r != last) {
                                  const int j = (int)p->run_step.size();
                                  p->run_step.push_back(steps + std::max(a, r_begin[r]) - a);
                                  for (int m = 0; m < nm; ++m) rvis[r].push_back(G * j + m);
                                  last = r;
                              }
                              ++r;
                          }
                          steps += b - a;
                      });
        }
        p->pool_run[H] = (int32_t)p->run_step.size();
        p->visits = G * (int)p->run_step.size();
        // bound for any split of the work list: a contiguous range meets one run per region it
        // meets; a rotated walk (at most one region boundary inside) adds at most two
        p->visit_cap = G * ((int)H + p->regions + 2 * (int)std::min<long long>(H, p->regions));
    } else {
        // one launch per region, each with its own small persistent grid
        const long long Cmax = (long long)p->num_sms * cps;
        p->pl_off.assign(p->regions + 1, 0);
        p->pl_ctas.assign(p->regions, 0);
        p->cta_item.clear();
        p->cta_visit.clear();
        int v = 0;
        for (int r = 0; r < p->regions; ++r) {
            const long long a = r_begin[r], b = r_begin[r + 1];
            const long long n = b - a;
            const int C = (int)std::max(0LL, std::min(Cmax, n));
            p->pl_off[r] = (int)p->cta_item.size();
            p->pl_ctas[r] = C;
            for (int c = 0; c <= C; ++c) p->cta_item.push_back(C ? a + n * c / C : a);
            for (int c = 0; c < C; ++c) {
                p->cta_visit.push_back(v);
                rvis[r].push_back(v++);
            }
            p->cta_visit.push_back(v);
        }
        p->pl_off[p->regions] = (int)p->cta_item.size();
        p->pools = 0;
        p->pool_size = 0;
        p->pool_item.assign(1, 0);
        p->pool_sweep.clear();
        p->pool_run.assign(1, 0);
        p->run_step.clear();
        p->visits = v;
        p->visit_cap = v;
        p->ctas = (int)Cmax;
    }
    p->region_visit_off.assign(p->regions + 1, 0);
    p->region_visits.clear();
    for (int r = 0; r < p->regions; ++r) {
        p->region_visit_off[r] = (int)p->region_visits.size();
        for (int v : rvis[r]) p->region_visits.push_back(v);
    }
    p->region_visit_off[p->regions] = (int)p->region_visits.size();
    p->cap = 2 * k + tile_b(p) * JW;
    // workspace layout
    size_t o = 0;
    p->off_probs = o; o = al(o + sizeof(ProbDev) * p->n);
    for (auto& h : p->P) {
        const ProbDev& pd = h.pd;
        h.off_orb = o; o = al(o + sizeof(double) * 4 * (size_t)pd.nOT);
        h.off_brow = o; o = al(o + sizeof(int32_t) * (size_t)pd.B);
        h.off_bap = o; o = al(o + sizeof(double) * (size_t)pd.B);
        h.off_bapq = o; o = al(o + sizeof(int32_t) * (size_t)pd.B);
        h.off_ps = o; o = al(o + sizeof(int64_t) * (pd.n_patch + 1));
        h.off_pos = o; o = al(o + sizeof(int32_t) * pd.S);
        h.off_vnq = o; o = al(o + sizeof(int32_t) * (size_t)pd.S * pd.Np);
        h.off_cq = o; o = al(o + sizeof(int32_t) * (size_t)pd.nOT * pd.Np);
        h.off_c64 = o; o = al(o + sizeof(double) * (size_t)pd.nOT * pd.Np);
        const size_t wsz = p->mode == BSH_MODE_PLAIN ? sizeof(double) : sizeof(float);
        h.off_w = o; o = al(o + wsz * (size_t)pd.S * pd.Np);
    }
    p->off_cta_item = o; o = al(o + sizeof(int64_t) * p->cta_item.size());
    p->off_cta_visit = o; o = al(o + sizeof(int32_t) * p->cta_visit.size());
    p->off_pool_item = o; o = al(o + sizeof(int64_t) * p->pool_item.size());
    p->off_pool_sweep = o; o = al(o + sizeof(int32_t) * std::max<size_t>(1, p->pool_sweep.size()));
    p->off_pool_run = o; o = al(o + sizeof(int32_t) * p->pool_run.size());
    p->off_run_step = o; o = al(o + sizeof(int64_t) * std::max<size_t>(1, p->run_step.size()));
    p->off_pool_next = o; o = al(o + sizeof(unsigned long long) * std::max(1, p->pools));
    p->off_vbuf = o; o = al(o + sizeof(Entry) * (size_t)p->visit_cap * p->cap);
    p->off_vcount = o; o = al(o + sizeof(int32_t) * (size_t)std::max(1, p->visit_cap));
    p->off_rprob = o; o = al(o + sizeof(int32_t) * p->regions);
    p->off_rvoff = o; o = al(o + sizeof(int32_t) * (p->regions + 1));
    p->off_rvis = o; o = al(o + sizeof(int32_t) * (size_t)std::max(1, p->visit_cap));
    p->off_scratch = o; o = al(o + sizeof(Entry) * (size_t)p->regions * k);
    p->off_dense = o; o = al(o + 2 * sizeof(void*) * p->n);
    p->ws_size = o;
    return BSH_OK;
}

template <class T>
cudaError_t up(void* dst, const T* src, size_t n, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    return cudaMemcpyAsync(dst, src, sizeof(T) * n, cudaMemcpyHostToDevice, st);
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult qr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &qr) ==
                cudaSuccess &&
            qr == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    });
    return fn;
}

int encode_bits_map(bsh_plan* p, int q) {
    const ProbHost& h = p->P[q];
    auto enc = get_encode();
    if (!enc) return BSH_ERR_CUDA;
    CUtensorMap* m = reinterpret_cast<CUtensorMap*>(p->maps.map[q]);
    cuuint64_t dims[2] = {(cuuint64_t)h.d.W, (cuuint64_t)h.d.N};
    cuuint64_t strides[1] = {(cuuint64_t)h.d.W * 4};
    cuuint32_t box[2] = {(cuuint32_t)p->wseg_max, (cuuint32_t)p->chunk};
    cuuint32_t es[2] = {1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, const_cast<uint32_t*>(h.d.bits), dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return BSH_ERR_ARG;
    // the fixed-point orbit table c_q [nOT][Np]: a box of crows rows x (chunk + pad) SFTs
    const ProbDev& pd = h.pd;
    CUtensorMap* mc = reinterpret_cast<CUtensorMap*>(p->maps.cmap[q]);
    cuuint64_t cdims[2] = {(cuuint64_t)pd.Np, (cuuint64_t)pd.nOT};
    cuuint64_t cstrides[1] = {(cuuint64_t)pd.Np * 4};
    cuuint32_t cbox[2] = {(cuuint32_t)count_c_stride(p->chunk), (cuuint32_t)pd.crows};
    r = enc(mc, CU_TENSOR_MAP_DATA_TYPE_INT32, 2, pd.c_q, cdims, cstrides, cbox, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? BSH_OK : BSH_ERR_ARG;
}

CountArgs count_args(bsh_plan* p, int dense) {
    CountArgs a{};
    a.probs = reinterpret_cast<const ProbDev*>(p->ws + p->off_probs);
    a.n_probs = p->n;
    a.cta_item = reinterpret_cast<const int64_t*>(p->ws + p->off_cta_item);
    a.cta_visit = reinterpret_cast<const int32_t*>(p->ws + p->off_cta_visit);
    a.pools = p->pools;
    a.pool_size = p->pool_size;
    a.pool_item = reinterpret_cast<const int64_t*>(p->ws + p->off_pool_item);
    a.pool_sweep = reinterpret_cast<const int32_t*>(p->ws + p->off_pool_sweep);
    a.pool_run = reinterpret_cast<const int32_t*>(p->ws + p->off_pool_run);
    a.run_step = reinterpret_cast<const int64_t*>(p->ws + p->off_run_step);
    a.pool_next = reinterpret_cast<unsigned long long*>(p->ws + p->off_pool_next);
    a.visit_buf = reinterpret_cast<Entry*>(p->ws + p->off_vbuf);
    a.visit_count = reinterpret_cast<int32_t*>(p->ws + p->off_vcount);
    a.cap = p->cap;
    a.top_k = p->top_k;
    a.dense = dense;
    a.dense_unw = reinterpret_cast<int32_t* const*>(p->ws + p->off_dense);
    a.dense_w = reinterpret_cast<float* const*>(p->ws + p->off_dense + sizeof(void*) * p->n);
    a.status = status_ptr();
    a.chunk = p->chunk;
    a.smem_bytes = p->smem;
    a.wseg_max = p->wseg_max;
    a.ot_max = p->ot_max;
    a.mode = p->mode;
    a.wrows = p->wrows;
    a.acc_mode = p->acc_mode;
    a.direct = p->direct;
    a.lut = p->lut;
    a.wait_polls = p->wait_polls;
    a.skip_stage = p->skip_stage;
    a.max_n = 0;
    for (auto& h : p->P) a.max_n = std::max(a.max_n, h.d.N);
    return a;
}

int run_count(bsh_plan* p, int dense, cudaStream_t st) {
    if (!p || !p->bound) return BSH_ERR_STATE;
    unsigned* sp = status_ptr();
    if (!sp) return BSH_ERR_CUDA;
    const ProbDev* dprobs = reinterpret_cast<const ProbDev*>(p->ws + p->off_probs);
    for (int q = 0; q < p->n; ++q) launch_tables(p->P[q].pd, dprobs + q, p->mode, sp, st);
    CountArgs a = count_args(p, dense);
    if (p->mode == BSH_MODE_BATCHED) {
        // every pool's item counter starts at 0; a visit buffer that neither CTA of its pool
        // opens (the other took all of the run's items) holds no entries
        cudaError_t e = cudaMemsetAsync(p->ws + p->off_pool_next, 0, sizeof(unsigned long long) * p->pools, st);
        if (e == cudaSuccess && !dense && p->visits > 0)
            e = cudaMemsetAsync(p->ws + p->off_vcount, 0, sizeof(int32_t) * p->visits, st);
        if (e != cudaSuccess) return cuda_fail(e);
        if (p->acc_mode == 2) launch_count_tc(a, p->maps, p->ctas, st);
        else launch_count(a, p->maps, p->ctas, p->threads, st);
    } else {
        for (int r = 0; r < p->regions; ++r) {
            if (p->pl_ctas[r] == 0) continue;
            CountArgs ar = a;
            ar.cta_item = a.cta_item + p->pl_off[r];
            ar.cta_visit = a.cta_visit + p->pl_off[r];
            launch_count(ar, p->maps, p->pl_ctas[r], p->threads, st);
        }
    }
    return cuda_fail(cudaGetLastError());
}

}  // namespace

namespace {
// Points the descriptors at the workspace under the current layout, encodes the
// TMA descriptors (peakgram rows, fixed-point orbit table) and uploads the small
// tables; synchronises `st`.
int upload_plan(bsh_plan* p, cudaStream_t st) {
    std::vector<ProbDev> hp(p->n);
    for (int q = 0; q < p->n; ++q) {
        ProbHost& h = p->P[q];
        ProbDev& pd = h.pd;
        const bsh_problem& d = h.d;
        pd.bits = d.bits;
        pd.rho = d.rho;
        pd.w = d.w;
        pd.sum_w = d.sum_w;
        pd.sum_w2 = d.sum_w2;
        pd.v = d.v;
        pd.t = d.t;
        pd.sky = d.sky;
        pd.orb = reinterpret_cast<const double*>(p->ws + h.off_orb);
        pd.brow = reinterpret_cast<const int32_t*>(p->ws + h.off_brow);
        pd.bap = reinterpret_cast<const double*>(p->ws + h.off_bap);
        pd.bapq = reinterpret_cast<const int32_t*>(p->ws + h.off_bapq);
        pd.patch_start = reinterpret_cast<const int64_t*>(p->ws + h.off_ps);
        pd.patch_of_s = reinterpret_cast<const int32_t*>(p->ws + h.off_pos);
        pd.vn_q = reinterpret_cast<int32_t*>(p->ws + h.off_vnq);
        pd.c_q = reinterpret_cast<int32_t*>(p->ws + h.off_cq);
        pd.c64 = reinterpret_cast<double*>(p->ws + h.off_c64);
        pd.crows = std::min(p->ot_max, pd.nOT);
        if (p->mode == BSH_MODE_PLAIN) {
            pd.w64 = reinterpret_cast<double*>(p->ws + h.off_w);
            pd.w32 = nullptr;
        } else {
            pd.w32 = reinterpret_cast<float*>(p->ws + h.off_w);
            pd.w64 = nullptr;
        }
        hp[q] = pd;
        cudaError_t e = cudaSuccess;
        e = e ? e : up(p->ws + h.off_orb, h.orb.data(), h.orb.size(), st);
        e = e ? e : up(p->ws + h.off_brow, h.brow.data(), h.brow.size(), st);
        e = e ? e : up(p->ws + h.off_bap, h.bap.data(), h.bap.size(), st);
        e = e ? e : up(p->ws + h.off_bapq, h.bapq.data(), h.bapq.size(), st);
        e = e ? e : up(p->ws + h.off_ps, h.ps.data(), h.ps.size(), st);
        e = e ? e : up(p->ws + h.off_pos, h.patch_of_s.data(), h.patch_of_s.size(), st);
        if (e) return BSH_ERR_CUDA;
        if (p->mode == BSH_MODE_BATCHED) {
            const int rc = encode_bits_map(p, q);
            if (rc) return rc;
        }
    }
    cudaError_t e = up(p->ws + p->off_probs, hp.data(), hp.size(), st);
    e = e ? e : up(p->ws + p->off_cta_item, p->cta_item.data(), p->cta_item.size(), st);
    e = e ? e : up(p->ws + p->off_cta_visit, p->cta_visit.data(), p->cta_visit.size(), st);
    e = e ? e : up(p->ws + p->off_pool_item, p->pool_item.data(), p->pool_item.size(), st);
    e = e ? e : up(p->ws + p->off_pool_sweep, p->pool_sweep.data(), p->pool_sweep.size(), st);
    e = e ? e : up(p->ws + p->off_pool_run, p->pool_run.data(), p->pool_run.size(), st);
    e = e ? e : up(p->ws + p->off_run_step, p->run_step.data(), p->run_step.size(), st);
    e = e ? e : up(p->ws + p->off_rprob, p->region_problem.data(), p->region_problem.size(), st);
    e = e ? e : up(p->ws + p->off_rvoff, p->region_visit_off.data(), p->region_visit_off.size(), st);
    e = e ? e : up(p->ws + p->off_rvis, p->region_visits.data(), p->region_visits.size(), st);
    e = e ? e : cudaMemsetAsync(p->ws + p->off_vcount, 0, sizeof(int32_t) * std::max(1, p->visits), st);
    e = e ? e : cudaStreamSynchronize(st);
    if (e) return BSH_ERR_CUDA;
    return BSH_OK;
}
}  // namespace

extern "C" {

int bsh_plan_bind(bsh_plan* p, void* workspace, size_t bytes, bsh_stream stream) {
    if (!p) return BSH_ERR_ARG;
    if (!workspace || bytes < p->ws_cap) return BSH_ERR_WORKSPACE;
    if (reinterpret_cast<uintptr_t>(workspace) % 256 != 0) return BSH_ERR_ARG;
    p->ws = static_cast<unsigned char*>(workspace);
    const int rc = upload_plan(p, (cudaStream_t)stream);
    if (rc) return rc;
    p->bound = true;
    return BSH_OK;
}

int bsh_autotune(bsh_plan* p, bsh_stream stream) {
    if (!p || !p->bound) return BSH_ERR_STATE;
    if (p->mode != BSH_MODE_BATCHED) return BSH_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const std::vector<int> ths = tune_threads(p), chs = tune_chunks(p);
    if (ths.size() * chs.size() <= 1) return BSH_OK;
    double best_rate = -1.0;
    int best_t = p->threads, best_c = p->chunk, best_a = p->acc_mode, best_o = p->one_cta, best_d = p->direct_tuned;
    // under the automatic choice both ways of forming the binary term are candidates
    const int n_dir = p->mode == BSH_MODE_BATCHED && p->direct_opt < 0 ? 2 : 1;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return BSH_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return BSH_ERR_CUDA;
    }
    int rc = BSH_OK;
    std::vector<long long> tried;
    for (int t : ths) {
        for (int c : chs) {
          for (int v = 0; v < 2 * n_dir; ++v) {
            // per way of forming the binary term, a second variant: the byte-table accumulation,
            // or for the per-term binary variant (predicated adds only) one CTA per SM with the
            // unshrunk stage
            const int am = v & 1;
            p->threads = t;
            p->chunk = c;
            if (n_dir == 2) p->direct_tuned = v >> 1;
            // the way build_schedule will take (p->wrows does not depend on the tile shape)
            const bool dir = p->direct_opt == 1 ||
                             (p->direct_opt < 0 && (p->direct_tuned >= 0 ? p->direct_tuned == 1 : p->wrows > 4));
            p->acc_mode = dir ? 0 : am;
            p->one_cta = dir ? am : 0;
            // a slice of the work list: about sixteen items per CTA of this shape
            const long long slice = (long long)p->num_sms * (512 / t) * 16;
            if (build_schedule(p, slice) != BSH_OK || p->ws_size > p->ws_cap) continue;
            // the stage may have been shrunk to fit shared memory: time each effective shape once
            const long long key = ((long long)t << 32) | ((long long)p->chunk << 4) | (p->direct << 2) |
                                  (p->acc_mode << 1) | p->one_cta;
            if (std::find(tried.begin(), tried.end(), key) != tried.end()) continue;
            tried.push_back(key);
            if ((rc = upload_plan(p, st)) != BSH_OK) break;
            // terms in the slice
            double terms = 0.0;
            for (long long it = 0; it < p->cta_item[p->ctas]; ++it) {
                int q = 0;
                while (q + 1 < p->n && it >= p->P[q + 1].pd.item_begin) ++q;
                const ProbDev& pd = p->P[q].pd;
                int fb, bt;
                item_fb_bt(p->P[q], it - pd.item_begin, &fb, &bt);
                const int tb = tile_b(p);
                const int nb = std::min(tb, pd.B - bt * tb);
                const int jb = std::min(pd.JB, pd.n_f0 - fb * pd.JB);
                terms += (double)nb * jb * pd.N;
            }
            if ((rc = run_count(p, 0, st)) != BSH_OK) break;   // warm-up
            float ms = 3.0e38f;
            for (int r = 0; r < 3 && rc == BSH_OK; ++r) {      // best of three
                cudaEventRecord(e0, st);
                rc = run_count(p, 0, st);
                cudaEventRecord(e1, st);
                if (rc != BSH_OK || cudaEventSynchronize(e1) != cudaSuccess) {
                    rc = rc ? rc : BSH_ERR_CUDA;
                    break;
                }
                float m = 0.f;
                cudaEventElapsedTime(&m, e0, e1);
                ms = std::min(ms, m);
            }
            if (rc != BSH_OK) break;
            const double rate = terms / (ms * 1e-3);
            if (rate > best_rate) {
                best_rate = rate;
                best_t = t;
                best_c = c;
                best_a = p->acc_mode;
                best_o = p->one_cta;
                best_d = p->direct_tuned;
            }
          }
          if (rc != BSH_OK) break;
        }
        if (rc != BSH_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    p->threads = best_t;
    p->chunk = best_c;
    p->acc_mode = best_a;
    p->one_cta = best_o;
    p->direct_tuned = best_d;
    const int rc2 = build_schedule(p);
    if (rc2 != BSH_OK) return rc2;
    const int rc3 = upload_plan(p, st);
    if (rc != BSH_OK) return rc;
    if (rc3 != BSH_OK) return rc3;
    p->tuned_rate = best_rate;
    return bsh_graph_reset(p);
}

int bsh_number_count(bsh_plan* p, bsh_stream stream) { return run_count(p, 0, (cudaStream_t)stream); }

int bsh_plan_tile(const bsh_plan* p, int* threads, int* sft_chunk, int* ctas) {
    if (!p || !threads || !sft_chunk || !ctas) return BSH_ERR_ARG;
    *threads = p->threads;
    *sft_chunk = p->chunk;
    *ctas = p->ctas;
    return BSH_OK;
}

int bsh_plan_set_accumulate(bsh_plan* p, int variant) {
    if (!p || variant < 0 || variant > 2) return BSH_ERR_ARG;
    if (variant == 2 && !tc_ok(p)) return BSH_ERR_ARG;
    p->acc_mode = variant;
    p->one_cta = 0;
    p->chunk = tune_chunks(p)[0];
    const int rc = build_schedule(p);
    if (rc) return rc;
    if (p->bound) {
        const int rc2 = upload_plan(p, nullptr);
        if (rc2) return rc2;
    }
    return bsh_graph_reset(p);
}

int bsh_plan_accumulate(const bsh_plan* p) { return p ? p->acc_mode : -1; }

int bsh_plan_set_direct(bsh_plan* p, int mode) {
    if (!p || mode < -1 || mode > 1) return BSH_ERR_ARG;
    p->direct_opt = mode;
    p->direct_tuned = -1;
    p->one_cta = 0;
    const int rc = build_schedule(p);
    if (rc) return rc;
    if (p->bound) {
        const int rc2 = upload_plan(p, nullptr);
        if (rc2) return rc2;
    }
    return bsh_graph_reset(p);
}

int bsh_plan_direct(const bsh_plan* p) { return p ? p->direct : -1; }

int bsh_plan_set_wait(bsh_plan* p, int polls, int skip_stage) {
    if (!p || polls < 0 || skip_stage < -1) return BSH_ERR_ARG;
    p->wait_polls = polls ? polls : kDefaultWaitPolls;
    p->skip_stage = skip_stage;
    return bsh_graph_reset(p);
}

int bsh_track_precision(bsh_plan* p, int problem, int s_begin, int s_end, unsigned long long* counts,
                        bsh_stream stream) {
    if (!p || !p->bound) return BSH_ERR_STATE;
    if (problem < 0 || problem >= p->n || !counts) return BSH_ERR_ARG;
    const ProbDev& hp = p->P[problem].pd;
    if (s_begin < 0 || s_end > hp.S || s_begin > s_end) return BSH_ERR_ARG;
    unsigned* sp = status_ptr();
    if (!sp) return BSH_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    const ProbDev* dprob = reinterpret_cast<const ProbDev*>(p->ws + p->off_probs) + problem;
    if (cudaMemsetAsync(counts, 0, 4 * sizeof(unsigned long long), st) != cudaSuccess) return BSH_ERR_CUDA;
    launch_tables(hp, dprob, p->mode, sp, st);
    launch_precision(dprob, s_begin, s_end, counts, st);
    return cuda_fail(cudaGetLastError());
}

int bsh_track_bins(bsh_plan* p, int problem, const int64_t* ids, int n, int32_t* bins, bsh_stream stream) {
    if (!p || !p->bound) return BSH_ERR_STATE;
    if (problem < 0 || problem >= p->n || n < 0 || (n > 0 && (!ids || !bins))) return BSH_ERR_ARG;
    unsigned* sp = status_ptr();
    if (!sp) return BSH_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    const ProbDev* dprob = reinterpret_cast<const ProbDev*>(p->ws + p->off_probs) + problem;
    launch_tables(p->P[problem].pd, dprob, p->mode, sp, st);
    launch_bins(dprob, ids, n, bins, sp, st);
    return cuda_fail(cudaGetLastError());
}

int bsh_cand_params(bsh_plan* p, int problem, const bsh_cand* cands, const int32_t* n_cands, int per_region,
                    int stat, const bsh_post_params* pp, double* params, double* sig, int32_t* valid,
                    bsh_stream stream) {
    if (!p || !p->bound) return BSH_ERR_STATE;
    if (problem < 0 || problem >= p->n || !cands || !n_cands || per_region <= 0 || (stat != 0 && stat != 1) ||
        !params || !sig || !valid)
        return BSH_ERR_ARG;
    const ProbHost& h = p->P[problem];
    const ProbDev* dprob = reinterpret_cast<const ProbDev*>(p->ws + p->off_probs) + problem;
    return launch_cand_params(dprob, h.pd.region_base, h.pd.n_patch, per_region, cands, n_cands, stat, pp, params,
                              sig, valid, (cudaStream_t)stream);
}

int bsh_count_dense(bsh_plan* p, int32_t* const* n_unw, float* const* n_w, bsh_stream stream) {
    if (!p || !p->bound) return BSH_ERR_STATE;
    if (!n_unw || !n_w) return BSH_ERR_ARG;
    std::vector<void*> ptrs(2 * p->n);
    for (int q = 0; q < p->n; ++q) {
        if (!n_unw[q] || !n_w[q]) return BSH_ERR_ARG;
        ptrs[q] = n_unw[q];
        ptrs[p->n + q] = n_w[q];
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemcpyAsync(p->ws + p->off_dense, ptrs.data(), sizeof(void*) * ptrs.size(), cudaMemcpyHostToDevice, st) !=
        cudaSuccess)
        return BSH_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return BSH_ERR_CUDA;
    return run_count(p, 1, st);
}

int bsh_toplist(bsh_plan* p, bsh_cand* out, int32_t* n_out, bsh_stream stream) {
    if (!p || !p->bound) return BSH_ERR_STATE;
    if (!out || !n_out) return BSH_ERR_ARG;
    MergeArgs a{};
    a.probs = reinterpret_cast<const ProbDev*>(p->ws + p->off_probs);
    a.n_probs = p->n;
    a.region_problem = reinterpret_cast<const int32_t*>(p->ws + p->off_rprob);
    a.region_visit_off = reinterpret_cast<const int32_t*>(p->ws + p->off_rvoff);
    a.region_visits = reinterpret_cast<const int32_t*>(p->ws + p->off_rvis);
    a.visit_buf = reinterpret_cast<const Entry*>(p->ws + p->off_vbuf);
    a.visit_count = reinterpret_cast<const int32_t*>(p->ws + p->off_vcount);
    a.cap = p->cap;
    a.top_k = p->top_k;
    a.scratch = reinterpret_cast<Entry*>(p->ws + p->off_scratch);
    a.out = out;
    a.n_out = n_out;
    a.status = status_ptr();
    launch_merge(a, p->regions, (cudaStream_t)stream);
    return cuda_fail(cudaGetLastError());
}

int bsh_power_sum(bsh_plan* p, bsh_cand* cands, const int32_t* n_cands, int n_cf, bsh_cand* final_list,
                  int32_t* n_final, bsh_stream stream) {
    if (!p || !p->bound) return BSH_ERR_STATE;
    if (!cands || !n_cands || !final_list || !n_final || n_cf < 1 || n_cf > p->top_k) return BSH_ERR_ARG;
    for (auto& h : p->P)
        if (!h.d.rho) return BSH_ERR_ARG;
    PowerArgs a{};
    a.probs = reinterpret_cast<const ProbDev*>(p->ws + p->off_probs);
    a.n_probs = p->n;
    a.region_problem = reinterpret_cast<const int32_t*>(p->ws + p->off_rprob);
    a.cands = cands;
    a.n_cands = n_cands;
    a.top_k = p->top_k;
    a.n_cf = n_cf;
    a.final_list = final_list;
    a.n_final = n_final;
    a.status = status_ptr();
    launch_power(a, p->regions, (cudaStream_t)stream);
    return cuda_fail(cudaGetLastError());
}

int bsh_power_sum_sft(bsh_plan* p2, const bsh_plan* p1, bsh_cand* cands, const int32_t* n_cands, int n_cf,
                      bsh_cand* final_list, int32_t* n_final, bsh_stream stream) {
    if (!p2 || !p1 || !p2->bound) return BSH_ERR_STATE;
    if (!cands || !n_cands || !final_list || !n_final || n_cf < 1 || n_cf > p1->top_k) return BSH_ERR_ARG;
    if (p2->mode != BSH_MODE_BATCHED || p2->n != p1->n || p2->regions != p1->regions) return BSH_ERR_ARG;
    for (int q = 0; q < p2->n; ++q) {
        const ProbHost& a = p1->P[q];
        const ProbHost& b = p2->P[q];
        // the same templates: sky count, patches, binary templates and f0 grid
        if (!b.d.rho || a.pd.S != b.pd.S || a.pd.B != b.pd.B || a.pd.n_f0 != b.pd.n_f0 || a.pd.F0 != b.pd.F0 ||
            a.ps != b.ps || a.orb != b.orb || a.brow != b.brow || a.bap != b.bap ||
            a.pd.region_base != b.pd.region_base)
            return BSH_ERR_ARG;
    }
    unsigned* sp = status_ptr();
    if (!sp) return BSH_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    const ProbDev* dprobs = reinterpret_cast<const ProbDev*>(p2->ws + p2->off_probs);
    for (int q = 0; q < p2->n; ++q) launch_tables(p2->P[q].pd, dprobs + q, p2->mode, sp, st);
    PowerArgs a{};
    a.probs = dprobs;
    a.n_probs = p2->n;
    a.region_problem = reinterpret_cast<const int32_t*>(p2->ws + p2->off_rprob);
    a.cands = cands;
    a.n_cands = n_cands;
    a.top_k = p1->top_k;
    a.n_cf = n_cf;
    a.final_list = final_list;
    a.n_final = n_final;
    a.status = sp;
    launch_power(a, p2->regions, st);
    return cuda_fail(cudaGetLastError());
}

int bsh_graph_reset(bsh_plan* p) {
    if (!p) return BSH_ERR_ARG;
    if (p->gexec) cudaGraphExecDestroy(p->gexec);
    if (p->graph) cudaGraphDestroy(p->graph);
    p->gexec = nullptr;
    p->graph = nullptr;
    return BSH_OK;
}

int bsh_graph_launch(bsh_plan* p, bsh_cand* cands, int32_t* n_cands, int n_cf, bsh_cand* final_list,
                     int32_t* n_final, bsh_stream stream) {
    if (!p || !p->bound) return BSH_ERR_STATE;
    cudaStream_t st = (cudaStream_t)stream;
    const void* args[6] = {cands, n_cands, final_list, n_final, nullptr, nullptr};
    if (p->gexec && (std::memcmp(args, p->g_args, sizeof(args)) != 0 || n_cf != p->g_ncf)) return BSH_ERR_STATE;
    if (!p->gexec) {
        // Record on a private stream: the caller's stream may be the legacy
        // default stream, which cannot be captured.  The graph is then
        // launched on the caller's stream.
        if (!p->cap_stream && cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
            return BSH_ERR_CUDA;
        cudaStream_t cs = p->cap_stream;
        if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return BSH_ERR_CUDA;
        int rc = bsh_number_count(p, (bsh_stream)cs);
        if (!rc) rc = bsh_toplist(p, cands, n_cands, (bsh_stream)cs);
        if (!rc) rc = bsh_power_sum(p, cands, n_cands, n_cf, final_list, n_final, (bsh_stream)cs);
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(cs, &g);
        if (rc || e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return rc ? rc : BSH_ERR_CUDA;
        }
        if (cudaGraphInstantiate(&p->gexec, g, 0) != cudaSuccess) {
            cudaGraphDestroy(g);
            return BSH_ERR_CUDA;
        }
        p->graph = g;
        std::memcpy(p->g_args, args, sizeof(args));
        p->g_ncf = n_cf;
    }
    return cuda_fail(cudaGraphLaunch(p->gexec, st));
}

}  // extern "C"

extern "C" int bsh_debug_track_windows(const bsh_problem* hp, const int32_t* query, int count,
                                       const uint32_t* row_bits, uint32_t* out, int32_t* path) {
    if (!hp || !query || count < 0 || !row_bits || !out || !path) return BSH_ERR_ARG;
    const bsh_problem& d = *hp;
    if (d.N <= 0 || d.K <= 0 || d.W < (d.K + 31) / 32 || !d.v || !d.t || !d.sky || d.n_f0 <= 0 ||
        !finite_pos(d.v_max))
        return BSH_ERR_ARG;
    if (uses_bank(d)) {
        if (d.n_bank <= 0 || !d.orbit || !d.bank_orbit || !d.bank_ap) return BSH_ERR_ARG;
        for (int b = 0; b < d.n_bank; ++b)
            if (d.bank_orbit[b] < 0 || d.bank_orbit[b] >= d.n_orbit) return BSH_ERR_ARG;
    } else if (!d.a_p || !d.Omega || !d.T_asc || d.n_ap <= 0 || d.n_Om <= 0 || d.n_T <= 0 || d.n_kappa < 0 ||
               d.n_eta < 0 || (d.n_kappa > 0 && !d.kappa) || (d.n_eta > 0 && !d.eta)) {
        return BSH_ERR_ARG;
    }
    bsh_plan tmp;
    tmp.threads = 256;
    ProbHost h;
    h.d = d;
    expand_binaries(h, d);
    const int64_t ps[2] = {0, d.S};
    h.ps.assign(ps, ps + 2);
    h.d.n_patch = 1;
    int rc = prepare_problem(&tmp, h);
    if (rc) return rc;
    const ProbDev& pd = h.pd;
    const FixedPoint& fp = pd.fp;
    const double sv = std::ldexp(1.0, fp.s_vn), sc = std::ldexp(1.0, fp.s_c);
    const int pos_max = 32 * d.W - 33;
    for (int e = 0; e < count; ++e) {
        const int s = query[4 * e], b = query[4 * e + 1], i = query[4 * e + 2], j0 = query[4 * e + 3];
        if (s < 0 || s >= d.S || b < 0 || b >= pd.B || i < 0 || i >= d.N || j0 < 0) return BSH_ERR_ARG;
        const double* n = d.sky + 3 * (size_t)s;
        const double* v = d.v + 3 * (size_t)i;
        volatile double t1 = v[0] * n[0], t2 = v[1] * n[1], t3 = v[2] * n[2];
        volatile double t12 = t1 + t2;
        const double vn = t12 + t3;
        const double* orow = h.orb.data() + 4 * (size_t)h.brow[b];
        const double Om = orow[0], Ta = orow[1], kap = orow[2], eta = orow[3];
        const int apq = h.bapq[b];
        volatile double dt = d.t[i] - Ta;
        volatile double arg = Om * dt;
        volatile double g = std::cos(arg);
        if (kap != 0.0 || eta != 0.0) {
            volatile double a2 = 2.0 * arg;
            volatile double kc = kap * std::cos(a2);
            volatile double es = eta * std::sin(a2);
            volatile double g1 = g + kc;
            g = g1 + es;
        }
        const double c = Om * g;
        const int vq = (int)std::nearbyint(vn * sv);
        const int cq = (int)std::nearbyint(c * sc);
        const int F2a = (int)std::llround(2.0 * d.F0) + 2 * j0;
        const int v0 = make_Z(F2a, vq, fp) - mulhi32(apq, make_C(F2a, cq, fp));
        const int v1 = make_Z(F2a + 62, vq, fp) - mulhi32(apq, make_C(F2a + 62, cq, fp));
        const int vr = make_Z(F2a + 30, vq, fp) - mulhi32(apq, make_C(F2a + 30, cq, fp));
        const uint32_t* row = row_bits + (size_t)e * d.W;
        const int pbase = pd.G0 + j0 - d.k_lo;
        const int pos = pbase + (vr >> fp.s_y);
        const double ap = h.bap[b];
        auto exact_o = [&](int j) -> int {
            volatile double apc = ap * c;
            volatile double D = vn - apc;
            const double F = d.F0 + (double)(j0 + j);
            volatile double FD = F * D;
            volatile double x = F + FD;
            volatile double xh = x + 0.5;
            return (int)((long long)std::floor(xh) - (long long)(pd.G0 + j0 + j));
        };
        if (fp_fast_ref(vr, fp_margin(vq, fp), fp.s_y) && (unsigned)pos <= (unsigned)pos_max) {
            out[e] = row_window(row, pos);
            path[e] = 0;
        } else {
            int pth = 0;
            bool bad = false;
            out[e] = fp_window_slow(v0, v1, pbase, pos_max, fp.s_y, fp.M, row, exact_o, &pth, &bad);
            path[e] = bad ? -1 : pth;
        }
    }
    return BSH_OK;
}

// ---------------------------------------------------------------------------
// Power sum without allocation: scratch in a static device array.
namespace {

__device__ __align__(256) unsigned char g_static_scratch[BSH_STATIC_SCRATCH_BYTES];

// Device address of g_static_scratch on the current device, looked up once per device.
unsigned char* static_scratch_ptr() {
    static std::mutex mu;
    static unsigned char* ptrs[64] = {nullptr};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(mu);
    if (!ptrs[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess) return nullptr;
        ptrs[dev] = static_cast<unsigned char*>(p);
    }
    return ptrs[dev];
}

// Compact grid arrays of a problem, staged in the static scratch.
struct GridDev {
    const double* a_p;     // [n_ap]
    const double* Om;      // [n_Om]
    const double* Ta;      // [n_Om][n_T]
    const double* kap;     // [n_kap] or NULL
    const double* eta;     // [n_eta] or NULL
    int n_ap, n_T, n_kap, n_eta;
};

// Writes the orbit rows and per-template (row, a_p) of a grid in its template order.
__global__ void static_expand(const ProbDev* probs, GridDev g) {
    const ProbDev& P = probs[0];
    const int nk = g.n_kap > 0 ? g.n_kap : 1, ne = g.n_eta > 0 ? g.n_eta : 1;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < P.nOT; r += gridDim.x * blockDim.x) {
        const int ie = r % ne, ik = (r / ne) % nk, t = r / ne / nk;   // t = iOm * n_T + iT
        double* o = const_cast<double*>(P.orb) + 4 * (size_t)r;
        o[0] = g.Om[t / g.n_T];
        o[1] = g.Ta[t];
        o[2] = g.kap ? g.kap[ik] : 0.0;
        o[3] = g.eta ? g.eta[ie] : 0.0;
    }
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < P.B; b += gridDim.x * blockDim.x) {
        const_cast<int32_t*>(P.brow)[b] = b / g.n_ap;
        const_cast<double*>(P.bap)[b] = g.a_p[b % g.n_ap];
    }
}

__global__ void static_bapq(const ProbDev* probs) {
    const ProbDev& P = probs[0];
    const double sc = ldexp(1.0, P.fp.s_a);
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < P.B; b += gridDim.x * blockDim.x)
        const_cast<int32_t*>(P.bapq)[b] = (int32_t)llrint(P.bap[b] * sc);
}

// One warp per listed template: Eq. (26) along the track (the plan's power kernel's sum).
__global__ void power_list_kernel(const ProbDev* probs, const int64_t* ids, int n, float* power, float* s_p,
                                  unsigned* status) {
    const int e = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (e >= n) return;
    const ProbDev& P = probs[0];
    const long long id = ids[e];
    const long long per_s = (long long)P.B * P.n_f0;
    if (id < 0 || id >= per_s * P.S) {
        if (lane == 0) {
            set_status(status, ST_ARG);
            power[e] = 0.f;
            s_p[e] = 0.f;
        }
        return;
    }
    const int s = (int)(id / per_s);
    const long long rem = id % per_s;
    const int b = (int)(rem / P.n_f0);
    const int j = (int)(rem % P.n_f0);
    const double v = warp_power_sum(P, s, b, j, status);
    if (lane == 0) {
        const double sw = P.sum_w[s], sw2 = P.sum_w2[s];
        power[e] = (float)v;
        s_p[e] = sw2 > 0.0 ? (float)((v - sw) / sqrt(sw2)) : 0.f;
    }
}

}  // namespace

extern "C" int bsh_power_sum_static(const bsh_problem* problem, const int64_t* template_ids, int n, float* power,
                                    float* s_p, bsh_stream stream) {
    if (!problem || n < 0 || (n > 0 && (!template_ids || !power || !s_p))) return BSH_ERR_ARG;
    const bsh_problem& d = *problem;
    int rc = validate_problem(d);
    if (rc) return rc;
    if (!d.rho) return BSH_ERR_ARG;
    if (n == 0) return BSH_OK;
    cudaStream_t st = (cudaStream_t)stream;
    ProbDev pd;
    std::memset(&pd, 0, sizeof(pd));
    pd.N = d.N;
    pd.Np = (d.N + 255) / 256 * 256;
    pd.K = d.K;
    pd.W = d.W;
    pd.k_lo = d.k_lo;
    pd.n_f0 = d.n_f0;
    pd.S = d.S;
    const bool bank = uses_bank(d);
    const int nk = std::max(1, d.n_kappa), ne = std::max(1, d.n_eta);
    const long long rows = bank ? d.n_orbit : (long long)d.n_Om * d.n_T * nk * ne;
    const long long B = binary_count(d);
    if (B > (1LL << 30) || (double)B * d.n_f0 * d.S > 9.0e18) return BSH_ERR_RANGE;
    pd.nOT = (int)rows;
    pd.B = (int)B;
    pd.w_dtype = d.w_dtype;
    pd.F0 = d.F0;
    pd.G0 = (int)std::floor(d.F0);
    pd.p_th = std::exp(-d.rho_th);
    pd.v_max = d.v_max;
    // largest a_p and |Omega g| bound, from the caller's arrays
    double ap_max = 0.0, Om_max = 0.0;
    if (bank) {
        for (int b = 0; b < d.n_bank; ++b) ap_max = std::max(ap_max, d.bank_ap[b]);
        for (int r = 0; r < d.n_orbit; ++r) {
            const double* o = d.orbit + 4 * (size_t)r;
            Om_max = std::max(Om_max, o[0] * (1.0 + std::fabs(o[2]) + std::fabs(o[3])));
        }
    } else {
        double km = 0.0, em = 0.0;
        for (int k = 0; k < d.n_ap; ++k) ap_max = std::max(ap_max, d.a_p[k]);
        for (int k = 0; k < d.n_Om; ++k) Om_max = std::max(Om_max, d.Omega[k]);
        for (int k = 0; k < d.n_kappa; ++k) km = std::max(km, std::fabs(d.kappa[k]));
        for (int k = 0; k < d.n_eta; ++k) em = std::max(em, std::fabs(d.eta[k]));
        Om_max *= 1.0 + km + em;
    }
    // the same fixed-point scales as a plan of this problem
    const int nb = (d.n_f0 + JW - 1) / JW;
    const int JB = (d.n_f0 + nb - 1) / nb;
    const int n_fb = (d.n_f0 + JB - 1) / JB;
    const double F_eval = d.F0 + (n_fb - 1) * JB + JW;
    rc = choose_fixed_point(F_eval, d.v_max, ap_max, Om_max, d.F0 - std::floor(d.F0), &pd.fp);
    if (rc) return rc;
    const double Fv_max = d.F0 + d.n_f0 - 1;
    const double yv = Fv_max * (d.v_max + ap_max * Om_max);
    const long long kmin = (long long)std::floor(d.F0 - yv + 0.5) - 1;
    const long long kmax = (long long)std::floor(Fv_max + yv + 0.5) + 1;
    if (kmin < d.k_lo || kmax >= (long long)d.k_lo + d.K) return BSH_ERR_RANGE;
    // scratch layout inside the static array
    size_t o = 0;
    const size_t off_pd = o; o = al(o + sizeof(ProbDev));
    const size_t off_orb = o; o = al(o + sizeof(double) * 4 * (size_t)rows);
    const size_t off_brow = o; o = al(o + sizeof(int32_t) * (size_t)B);
    const size_t off_bap = o; o = al(o + sizeof(double) * (size_t)B);
    const size_t off_bapq = o; o = al(o + sizeof(int32_t) * (size_t)B);
    size_t off_gap = 0, off_gOm = 0, off_gTa = 0, off_gk = 0, off_ge = 0;
    if (!bank) {
        off_gap = o; o = al(o + sizeof(double) * d.n_ap);
        off_gOm = o; o = al(o + sizeof(double) * d.n_Om);
        off_gTa = o; o = al(o + sizeof(double) * (size_t)d.n_Om * d.n_T);
        off_gk = o; o = al(o + sizeof(double) * nk);
        off_ge = o; o = al(o + sizeof(double) * ne);
    }
    const size_t off_vnq = o; o = al(o + sizeof(int32_t) * (size_t)d.S * pd.Np);
    const size_t off_w = o; o = al(o + sizeof(float) * (size_t)d.S * pd.Np);
    const size_t off_cq = o; o = al(o + sizeof(int32_t) * (size_t)rows * pd.Np);
    const size_t off_c64 = o; o = al(o + sizeof(double) * (size_t)rows * pd.Np);
    if (o > (size_t)BSH_STATIC_SCRATCH_BYTES) return BSH_ERR_WORKSPACE;
    unsigned char* base = static_scratch_ptr();
    unsigned* sp = status_ptr();
    if (!base || !sp) return BSH_ERR_CUDA;
    pd.bits = d.bits;
    pd.rho = d.rho;
    pd.w = d.w;
    pd.sum_w = d.sum_w;
    pd.sum_w2 = d.sum_w2;
    pd.v = d.v;
    pd.t = d.t;
    pd.sky = d.sky;
    pd.orb = reinterpret_cast<const double*>(base + off_orb);
    pd.brow = reinterpret_cast<const int32_t*>(base + off_brow);
    pd.bap = reinterpret_cast<const double*>(base + off_bap);
    pd.bapq = reinterpret_cast<const int32_t*>(base + off_bapq);
    pd.vn_q = reinterpret_cast<int32_t*>(base + off_vnq);
    pd.w32 = reinterpret_cast<float*>(base + off_w);
    pd.c_q = reinterpret_cast<int32_t*>(base + off_cq);
    pd.c64 = reinterpret_cast<double*>(base + off_c64);
    cudaError_t e = cudaMemcpyAsync(base + off_pd, &pd, sizeof(pd), cudaMemcpyHostToDevice, st);
    GridDev g{};
    if (bank) {
        e = e ? e : cudaMemcpyAsync(base + off_orb, d.orbit, sizeof(double) * 4 * (size_t)rows,
                                    cudaMemcpyHostToDevice, st);
        e = e ? e : cudaMemcpyAsync(base + off_brow, d.bank_orbit, sizeof(int32_t) * (size_t)B,
                                    cudaMemcpyHostToDevice, st);
        e = e ? e : cudaMemcpyAsync(base + off_bap, d.bank_ap, sizeof(double) * (size_t)B, cudaMemcpyHostToDevice,
                                    st);
    } else {
        e = e ? e : cudaMemcpyAsync(base + off_gap, d.a_p, sizeof(double) * d.n_ap, cudaMemcpyHostToDevice, st);
        e = e ? e : cudaMemcpyAsync(base + off_gOm, d.Omega, sizeof(double) * d.n_Om, cudaMemcpyHostToDevice, st);
        e = e ? e : cudaMemcpyAsync(base + off_gTa, d.T_asc, sizeof(double) * (size_t)d.n_Om * d.n_T,
                                    cudaMemcpyHostToDevice, st);
        if (d.n_kappa > 0)
            e = e ? e : cudaMemcpyAsync(base + off_gk, d.kappa, sizeof(double) * d.n_kappa, cudaMemcpyHostToDevice, st);
        if (d.n_eta > 0)
            e = e ? e : cudaMemcpyAsync(base + off_ge, d.eta, sizeof(double) * d.n_eta, cudaMemcpyHostToDevice, st);
        g.a_p = reinterpret_cast<const double*>(base + off_gap);
        g.Om = reinterpret_cast<const double*>(base + off_gOm);
        g.Ta = reinterpret_cast<const double*>(base + off_gTa);
        g.kap = d.n_kappa > 0 ? reinterpret_cast<const double*>(base + off_gk) : nullptr;
        g.eta = d.n_eta > 0 ? reinterpret_cast<const double*>(base + off_ge) : nullptr;
        g.n_ap = d.n_ap;
        g.n_T = d.n_T;
        g.n_kap = d.n_kappa;
        g.n_eta = d.n_eta;
    }
    if (e) return BSH_ERR_CUDA;
    const ProbDev* dpd = reinterpret_cast<const ProbDev*>(base + off_pd);
    if (!bank) static_expand<<<64, 256, 0, st>>>(dpd, g);
    static_bapq<<<64, 256, 0, st>>>(dpd);
    launch_tables(pd, dpd, BSH_MODE_BATCHED, sp, st);
    const int warps = 8;
    power_list_kernel<<<(n + warps - 1) / warps, warps * 32, 0, st>>>(dpd, template_ids, n, power, s_p, sp);
    return cuda_fail(cudaGetLastError());
}
