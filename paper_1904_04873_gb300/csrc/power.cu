// Stage 2 (Sec. IV.C, Eq. (26)): for every toplist candidate, the weighted sum of
// normalised powers along its exact track, P = sum_i w_i rho_i[k_i], and
// s_P = (P - sum w)/sqrt(sum w^2); then each region is re-ranked by s_P and
// cut to N_CF.  The bin of each term comes from the same fixed-point track as
// the count (exact FP64 expression near rounding boundaries).
#include "bsh_internal.cuh"
#include "select.cuh"

namespace bsh {
namespace {

constexpr int PW = 8;        // warps per block in the power kernel
constexpr int RT = 512;      // threads of the re-rank kernel

__global__ void __launch_bounds__(PW * 32) power_kernel(const PowerArgs a) {
    const int r = blockIdx.y;
    const int e = blockIdx.x * PW + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (e >= a.n_cands[r]) return;                       // warp-uniform
    bsh_cand* c = a.cands + (size_t)r * a.top_k + e;
    const int q = a.region_problem[r];
    const ProbDev& P = a.probs[q];
    const long long id = c->template_id;
    const long long per_s = (long long)P.B * P.n_f0;
    const int s = (int)(id / per_s);
    const long long rem = id % per_s;
    const int b = (int)(rem / P.n_f0);
    const int j = (int)(rem % P.n_f0);
    const double tot = warp_power_sum(P, s, b, j, a.status);
    if (lane == 0) {
        const double sw = P.sum_w[s], sw2 = P.sum_w2[s];
        c->power = (float)tot;
        c->s_p = sw2 > 0.0 ? (float)((tot - sw) / sqrt(sw2)) : 0.f;
    }
}

__global__ void __launch_bounds__(RT) rerank_kernel(const PowerArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int r = blockIdx.x;
    const int n = a.n_cands[r];
    const int q = a.region_problem[r];
    const ProbDev& P = a.probs[q];
    const int patch = r - P.region_base;
    const long long gbase = P.patch_start[patch] * (long long)P.B * P.n_f0;
    int n2 = 1;
    while (n2 < n) n2 <<= 1;
    unsigned long long* key = reinterpret_cast<unsigned long long*>(smem);
    int* idx = reinterpret_cast<int*>(smem + (size_t)n2 * 8);
    const bsh_cand* c = a.cands + (size_t)r * a.top_k;
    for (int e = threadIdx.x; e < n2; e += RT) {
        unsigned long long k = 0ull;
        if (e < n) k = make_key(c[e].s_p, (uint32_t)(c[e].template_id - gbase));
        key[e] = k;
        idx[e] = e;
    }
    cta_bitonic_desc<RT>(key, idx, n2);
    const int m = n < a.n_cf ? n : a.n_cf;
    bsh_cand* out = a.final_list + (size_t)r * a.n_cf;
    for (int e = threadIdx.x; e < m; e += RT) out[e] = c[idx[e]];
    if (threadIdx.x == 0) a.n_final[r] = m;
}

}  // namespace

void launch_power(const PowerArgs& a, int regions, cudaStream_t st) {
    if (regions <= 0) return;
    dim3 grid((a.top_k + PW - 1) / PW, regions);
    power_kernel<<<grid, PW * 32, 0, st>>>(a);
    int n2 = 1;
    while (n2 < a.top_k) n2 <<= 1;
    const int smem = n2 * 12;
    static int s_rerank = 0;
    ensure_smem(rerank_kernel, smem, &s_rerank);
    rerank_kernel<<<regions, RT, smem, st>>>(a);
}

}  // namespace bsh
