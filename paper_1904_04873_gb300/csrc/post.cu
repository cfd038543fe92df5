// Post-processing of the toplists (Sec. V.E): candidate parameters, the distance of
// Eq. (44) with the resolutions of Eq. (30)-(32) and Sec. V.B averaged over the two
// candidates, coincidences between two lists (option A), clustering as connected
// components of the threshold graph (lock-free union-find that always links the larger
// root under the smaller, so each component's root is its smallest index), the
// option-B cut around each cluster's most significant member, significance-weighted
// centroids and the band's most significant cluster.
//
// Every threshold decision compares a squared distance accumulated in FP64 in a fixed
// order (one term per parameter, each rounded separately, no fused multiply-add); the
// terms are non-negative, so a partial sum that already reaches the threshold decides.
#include <cmath>
#include <cstdint>
#include <cstring>

#include "bsh_internal.cuh"

namespace bsh {
namespace {

constexpr double PI = 3.14159265358979323846;
constexpr int TB = 128;          // candidates per tile of the pair kernels

struct PostConst {
    double T_c, T_obs, v_over_c, P_F, m_a, m_Om, m_t;
    double s6a, s72o, s6t;       // sqrt(6 m_a), sqrt(72 m_Om), sqrt(6 m_t)
    double D2;                   // squared threshold of the pair kernel
    double C2;                   // squared cut distance (<= 0: no cut)
};

PostConst make_const(const bsh_post_params& pp, double D) {
    PostConst c;
    c.T_c = pp.T_c;
    c.T_obs = pp.T_obs;
    c.v_over_c = pp.v_over_c;
    c.P_F = pp.P_F;
    c.m_a = pp.m_a;
    c.m_Om = pp.m_Om;
    c.m_t = pp.m_t;
    c.s6a = std::sqrt(6.0 * pp.m_a);
    c.s72o = std::sqrt(72.0 * pp.m_Om);
    c.s6t = std::sqrt(6.0 * pp.m_t);
    c.D2 = D * D;
    c.C2 = pp.d_cut > 0.0 ? pp.d_cut * pp.d_cut : -1.0;
    return c;
}

__device__ __forceinline__ unsigned long long order64(double x) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    return (u & 0x8000000000000000ull) ? ~u : (u | 0x8000000000000000ull);
}

// Resolutions at one candidate: delta f, delta theta (x, y), delta a_p, delta Omega, delta t_asc.
__global__ void res_kernel(const double* __restrict__ p, int n, PostConst c, double* __restrict__ res) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double* q = p + 6 * (size_t)i;
        const double f = q[0], a = q[3], Om = q[4];
        const double ptf = __dmul_rn(__dmul_rn(PI, c.T_c), f);
        const double d_th = __ddiv_rn(1.0, __dmul_rn(__dmul_rn(__dmul_rn(c.v_over_c, c.T_c), f), c.P_F));
        double* r = res + 6 * (size_t)i;
        r[0] = __ddiv_rn(1.0, c.T_c);
        r[1] = d_th;
        r[2] = d_th;
        r[3] = __ddiv_rn(c.s6a, __dmul_rn(ptf, Om));
        r[4] = __ddiv_rn(c.s72o, __dmul_rn(__dmul_rn(__dmul_rn(ptf, a), Om), c.T_obs));
        r[5] = __ddiv_rn(c.s6t, __dmul_rn(__dmul_rn(__dmul_rn(ptf, a), Om), Om));
    }
}

// Squared distance with an early exit once the partial sum reaches lim.
__device__ __forceinline__ double dist2(const double* pi, const double* ri, const double* pj, const double* rj,
                                        double lim) {
    double d2 = 0.0;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const double r = __dmul_rn(0.5, __dadd_rn(ri[k], rj[k]));
        const double q = __ddiv_rn(__dsub_rn(pi[k], pj[k]), r);
        d2 = __dadd_rn(d2, __dmul_rn(q, q));
        if (d2 >= lim) return d2;
    }
    return d2;
}

// Root of x: parents only ever point to smaller indices, so the walk ends within x steps.
__device__ __forceinline__ int uf_find(const int* parent, int x) {
    for (int it = 0; it <= x + 1; ++it) {
        const int p = __ldcg(parent + x);
        if (p == x) return x;
        x = p;
    }
    return x;
}

__device__ void uf_union(int* parent, int a, int b) {
    for (int it = 0; it < (1 << 22); ++it) {
        a = uf_find(parent, a);
        b = uf_find(parent, b);
        if (a == b) return;
        if (a < b) {
            const int t = a;
            a = b;
            b = t;
        }
        const int old = atomicCAS(parent + a, a, b);   // link the larger root under the smaller
        if (old == a) return;
        a = old;                                       // a was linked meanwhile: retry from there
    }
}

__global__ void init_kernel(const int32_t* __restrict__ valid, int n, int32_t* label, int32_t* keep, double* centroid,
                            double* csig, unsigned long long* topkey, int* topidx, double* wsum, double* psum,
                            int* cnt) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        label[i] = valid[i] ? i : -1;
        keep[i] = 0;
        csig[i] = 0.0;
        topkey[i] = 0ull;
        topidx[i] = 0x7fffffff;
        wsum[i] = 0.0;
        cnt[i] = 0;
        for (int k = 0; k < 6; ++k) {
            centroid[6 * (size_t)i + k] = 0.0;
            psum[6 * (size_t)i + k] = 0.0;
        }
    }
}

// Edges of the threshold graph over tiles (i block, j block >= i block), unioned as found.
__global__ void __launch_bounds__(TB) pair_union_kernel(const double* __restrict__ p, const double* __restrict__ res,
                                                        const int32_t* __restrict__ valid, int n, PostConst c,
                                                        int32_t* parent) {
    if (blockIdx.x < blockIdx.y) return;
    __shared__ double sp[TB * 6], sr[TB * 6];
    __shared__ int sv[TB];
    const int j0 = blockIdx.x * TB;
    for (int e = threadIdx.x; e < TB * 6; e += TB) {
        const int j = j0 + e / 6;
        sp[e] = j < n ? p[6 * (size_t)j0 + e] : 0.0;
        sr[e] = j < n ? res[6 * (size_t)j0 + e] : 1.0;
    }
    sv[threadIdx.x] = (j0 + (int)threadIdx.x < n) ? valid[j0 + threadIdx.x] : 0;
    __syncthreads();
    const int i = blockIdx.y * TB + threadIdx.x;
    if (i >= n || !valid[i]) return;
    double pi[6], ri[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        pi[k] = p[6 * (size_t)i + k];
        ri[k] = res[6 * (size_t)i + k];
    }
    for (int jj = 0; jj < TB; ++jj) {
        const int j = j0 + jj;
        if (j <= i || !sv[jj]) continue;
        if (dist2(pi, ri, sp + 6 * jj, sr + 6 * jj, c.D2) < c.D2) uf_union(parent, i, j);
    }
}

__global__ void flatten_kernel(int32_t* label, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        if (label[i] >= 0) label[i] = uf_find(label, i);
}

__global__ void top_key_kernel(const double* __restrict__ sig, const int32_t* __restrict__ label, int n,
                               unsigned long long* topkey) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        if (label[i] >= 0) atomicMax(topkey + label[i], order64(sig[i]));
}

__global__ void top_idx_kernel(const double* __restrict__ sig, const int32_t* __restrict__ label, int n,
                               const unsigned long long* __restrict__ topkey, int* topidx) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int r = label[i];
        if (r >= 0 && order64(sig[i]) == topkey[r]) atomicMin(topidx + r, i);
    }
}

// Option-B cut and the centroid sums of the kept members.
__global__ void cut_kernel(const double* __restrict__ p, const double* __restrict__ res,
                           const double* __restrict__ sig, const int32_t* __restrict__ label, int n, PostConst c,
                           const int* __restrict__ topidx, int32_t* keep, double* centroid, double* csig,
                           double* wsum, double* psum, int* cnt) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int r = label[i];
        if (r < 0) continue;
        const int t = topidx[r];
        bool k = true;
        if (c.C2 > 0.0) {
            const double d2 = dist2(p + 6 * (size_t)t, res + 6 * (size_t)t, p + 6 * (size_t)i, res + 6 * (size_t)i,
                                    INFINITY);
            k = d2 <= c.C2;
        }
        keep[i] = k ? 1 : 0;
        if (!k) continue;
        const double s = sig[i];
        const double w = s > 0.0 ? s : 0.0;
        atomicAdd(csig + r, s);
        atomicAdd(wsum + r, w);
        atomicAdd(cnt + r, 1);
        for (int q = 0; q < 6; ++q) {
            const double x = p[6 * (size_t)i + q];
            atomicAdd(centroid + 6 * (size_t)r + q, __dmul_rn(w, x));
            atomicAdd(psum + 6 * (size_t)r + q, x);
        }
    }
}

__global__ void finalize_kernel(const int32_t* __restrict__ label, int n, double* centroid, double* csig,
                                const double* __restrict__ wsum, const double* __restrict__ psum,
                                const int* __restrict__ cnt, unsigned long long* bestkey) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double* cen = centroid + 6 * (size_t)i;
        if (label[i] != i) {
            for (int q = 0; q < 6; ++q) cen[q] = __longlong_as_double(0x7ff8000000000000ll);
            csig[i] = 0.0;
            continue;
        }
        const double sw = wsum[i];
        for (int q = 0; q < 6; ++q)
            cen[q] = sw > 0.0 ? __ddiv_rn(cen[q], sw) : __ddiv_rn(psum[6 * (size_t)i + q], (double)cnt[i]);
        atomicMax(bestkey, order64(csig[i]));
    }
}

__global__ void best_kernel(const int32_t* __restrict__ label, int n, const double* __restrict__ csig,
                            const unsigned long long* __restrict__ bestkey, int* bestidx) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        if (label[i] == i && order64(csig[i]) == *bestkey) atomicMin(bestidx, i);
}

__global__ void best_out_kernel(const int* __restrict__ bestidx, int n, int32_t* best) {
    best[0] = (*bestidx >= 0 && *bestidx < n) ? *bestidx : -1;
}

// Option A: pairs of list A and list B closer than the threshold.
__global__ void __launch_bounds__(TB) coinc_kernel(const double* __restrict__ pa, const double* __restrict__ ra,
                                                   const double* __restrict__ sa, const int32_t* __restrict__ va,
                                                   int na, const double* __restrict__ pb,
                                                   const double* __restrict__ rb, const double* __restrict__ sb,
                                                   const int32_t* __restrict__ vb, int nb, PostConst c,
                                                   int32_t* pairs, double* cen, double* sig, int cap,
                                                   int32_t* n_pairs) {
    __shared__ double sp[TB * 6], sr[TB * 6];
    __shared__ int sv[TB];
    const int j0 = blockIdx.x * TB;
    for (int e = threadIdx.x; e < TB * 6; e += TB) {
        const int j = j0 + e / 6;
        sp[e] = j < nb ? pb[6 * (size_t)j0 + e] : 0.0;
        sr[e] = j < nb ? rb[6 * (size_t)j0 + e] : 1.0;
    }
    sv[threadIdx.x] = (j0 + (int)threadIdx.x < nb) ? vb[j0 + threadIdx.x] : 0;
    __syncthreads();
    const int i = blockIdx.y * TB + threadIdx.x;
    if (i >= na || !va[i]) return;
    double pi[6], ri[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        pi[k] = pa[6 * (size_t)i + k];
        ri[k] = ra[6 * (size_t)i + k];
    }
    for (int jj = 0; jj < TB; ++jj) {
        const int j = j0 + jj;
        if (j >= nb || !sv[jj]) continue;
        if (dist2(pi, ri, sp + 6 * jj, sr + 6 * jj, c.D2) >= c.D2) continue;
        const int slot = atomicAdd(n_pairs, 1);
        if (slot >= cap) continue;
        pairs[2 * (size_t)slot] = i;
        pairs[2 * (size_t)slot + 1] = j;
        const double s_a = sa[i], s_b = sb[j];
        const double wa = s_a > 0.0 ? s_a : 0.0, wb = s_b > 0.0 ? s_b : 0.0;
        const double sw = __dadd_rn(wa, wb);
        for (int k = 0; k < 6; ++k) {
            const double x = pi[k], y = sp[6 * jj + k];
            cen[6 * (size_t)slot + k] = sw > 0.0 ? __ddiv_rn(__dadd_rn(__dmul_rn(wa, x), __dmul_rn(wb, y)), sw)
                                                 : __dmul_rn(0.5, __dadd_rn(x, y));
        }
        sig[slot] = __dadd_rn(s_a, s_b);
    }
}

// Parameters of the candidates of one problem's regions.
__global__ void cand_params_kernel(const ProbDev* __restrict__ probs, int first_region, int n_rows, int per_region,
                                   const bsh_cand* __restrict__ cands, const int32_t* __restrict__ n_cands, int stat,
                                   double T_c, double ce, double se, double* params, double* sig, int32_t* valid) {
    const ProbDev& P = probs[0];
    for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < n_rows; row += gridDim.x * blockDim.x) {
        const int pch = row / per_region, e = row % per_region;
        const int r = first_region + pch;
        double* o = params + 6 * (size_t)row;
        const long long per_s = (long long)P.B * P.n_f0;
        const bsh_cand& cd = cands[(size_t)r * per_region + e];
        const long long id = cd.template_id;
        const bool ok = e < n_cands[r] && id >= 0 && id < per_s * P.S;
        valid[row] = ok ? 1 : 0;
        if (!ok) {
            for (int k = 0; k < 6; ++k) o[k] = 0.0;
            sig[row] = 0.0;
            continue;
        }
        const int s = (int)(id / per_s);
        const long long rem = id % per_s;
        const int b = (int)(rem / P.n_f0);
        const int j = (int)(rem % P.n_f0);
        const double* n = P.sky + 3 * (size_t)s;
        const double* orow = P.orb + 4 * (size_t)P.brow[b];
        o[0] = __ddiv_rn(__dadd_rn(P.F0, (double)j), T_c);
        o[1] = n[0];
        o[2] = __dadd_rn(__dmul_rn(ce, n[1]), __dmul_rn(se, n[2]));
        o[3] = P.bap[b];
        o[4] = orow[0];
        o[5] = orow[1];
        sig[row] = stat ? (double)cd.s_p : (double)cd.s_h;
    }
}

size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

int blocks_for(long long n) {
    long long b = (n + 255) / 256;
    if (b < 1) b = 1;
    if (b > 4096) b = 4096;
    return (int)b;
}

bool params_ok(const bsh_post_params* pp) {
    if (!pp) return false;
    const double v[] = {pp->T_c, pp->T_obs, pp->v_over_c, pp->P_F, pp->m_a, pp->m_Om, pp->m_t};
    for (double x : v)
        if (!(x > 0.0) || !std::isfinite(x)) return false;
    return std::isfinite(pp->obliquity) && std::isfinite(pp->d_cut) && pp->d_cluster > 0.0 && pp->d_coinc > 0.0 &&
           std::isfinite(pp->d_cluster) && std::isfinite(pp->d_coinc);
}

}  // namespace

int launch_cand_params(const ProbDev* dprob, int first_region, int n_patch, int per_region, const bsh_cand* cands,
                       const int32_t* n_cands, int stat, const bsh_post_params* pp, double* params, double* sig,
                       int32_t* valid, cudaStream_t st) {
    if (!params_ok(pp)) return BSH_ERR_ARG;
    const long long n = (long long)n_patch * per_region;
    if (n <= 0) return BSH_OK;
    cand_params_kernel<<<blocks_for(n), 256, 0, st>>>(dprob, first_region, (int)n, per_region, cands, n_cands, stat,
                                                      pp->T_c, std::cos(pp->obliquity), std::sin(pp->obliquity),
                                                      params, sig, valid);
    return cudaGetLastError() == cudaSuccess ? BSH_OK : BSH_ERR_CUDA;
}

}  // namespace bsh

using namespace bsh;

extern "C" size_t bsh_cluster_workspace(int n) {
    if (n <= 0) return 0;
    const size_t m = (size_t)n;
    return al256(m * 48) + al256(m * 8) + al256(m * 4) + al256(m * 8) + al256(m * 48) + al256(m * 4) + al256(16);
}

extern "C" int bsh_cluster(const double* params, const double* sig, const int32_t* valid, int n,
                           const bsh_post_params* pp, void* work, size_t work_bytes, int32_t* label, int32_t* keep,
                           double* centroid, double* csig, int32_t* best, bsh_stream stream) {
    if (n < 0 || n > (1 << 20) || !params_ok(pp)) return BSH_ERR_ARG;
    if (n > 0 && (!params || !sig || !valid || !label || !keep || !centroid || !csig || !best)) return BSH_ERR_ARG;
    if (!best) return BSH_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (n == 0) {
        const int32_t none = -1;
        return cudaMemcpyAsync(best, &none, sizeof(none), cudaMemcpyHostToDevice, st) == cudaSuccess ? BSH_OK
                                                                                                     : BSH_ERR_CUDA;
    }
    if (!work || work_bytes < bsh_cluster_workspace(n)) return BSH_ERR_WORKSPACE;
    const size_t m = (size_t)n;
    unsigned char* w = static_cast<unsigned char*>(work);
    size_t o = 0;
    double* res = reinterpret_cast<double*>(w + o); o += al256(m * 48);
    unsigned long long* topkey = reinterpret_cast<unsigned long long*>(w + o); o += al256(m * 8);
    int* topidx = reinterpret_cast<int*>(w + o); o += al256(m * 4);
    double* wsum = reinterpret_cast<double*>(w + o); o += al256(m * 8);
    double* psum = reinterpret_cast<double*>(w + o); o += al256(m * 48);
    int* cnt = reinterpret_cast<int*>(w + o); o += al256(m * 4);
    unsigned long long* bestkey = reinterpret_cast<unsigned long long*>(w + o);
    int* bestidx = reinterpret_cast<int*>(w + o + 8);
    const PostConst c = make_const(*pp, pp->d_cluster);
    const int nb = blocks_for(n);
    cudaError_t e = cudaMemsetAsync(bestkey, 0, 8, st);
    e = e ? e : cudaMemsetAsync(bestidx, 0x7f, 4, st);   // 0x7f7f7f7f: above every index
    if (e) return BSH_ERR_CUDA;
    res_kernel<<<nb, 256, 0, st>>>(params, n, c, res);
    init_kernel<<<nb, 256, 0, st>>>(valid, n, label, keep, centroid, csig, topkey, topidx, wsum, psum, cnt);
    const unsigned tiles = (unsigned)((n + TB - 1) / TB);
    pair_union_kernel<<<dim3(tiles, tiles), TB, 0, st>>>(params, res, valid, n, c, label);
    flatten_kernel<<<nb, 256, 0, st>>>(label, n);
    top_key_kernel<<<nb, 256, 0, st>>>(sig, label, n, topkey);
    top_idx_kernel<<<nb, 256, 0, st>>>(sig, label, n, topkey, topidx);
    cut_kernel<<<nb, 256, 0, st>>>(params, res, sig, label, n, c, topidx, keep, centroid, csig, wsum, psum, cnt);
    finalize_kernel<<<nb, 256, 0, st>>>(label, n, centroid, csig, wsum, psum, cnt, bestkey);
    best_kernel<<<nb, 256, 0, st>>>(label, n, csig, bestkey, bestidx);
    best_out_kernel<<<1, 1, 0, st>>>(bestidx, n, best);
    return cudaGetLastError() == cudaSuccess ? BSH_OK : BSH_ERR_CUDA;
}

extern "C" size_t bsh_coincidence_workspace(int na, int nb) {
    if (na < 0 || nb < 0) return 0;
    return al256((size_t)na * 48) + al256((size_t)nb * 48);
}

extern "C" int bsh_coincidences(const double* pa, const double* sa, const int32_t* va, int na, const double* pb,
                                const double* sb, const int32_t* vb, int nb, const bsh_post_params* pp, void* work,
                                size_t work_bytes, int32_t* pairs, double* centroid, double* sig, int cap,
                                int32_t* n_pairs, bsh_stream stream) {
    if (na < 0 || nb < 0 || na > (1 << 20) || nb > (1 << 20) || cap < 0 || !n_pairs || !params_ok(pp))
        return BSH_ERR_ARG;
    if ((na > 0 && (!pa || !sa || !va)) || (nb > 0 && (!pb || !sb || !vb))) return BSH_ERR_ARG;
    if (cap > 0 && (!pairs || !centroid || !sig)) return BSH_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(n_pairs, 0, sizeof(int32_t), st) != cudaSuccess) return BSH_ERR_CUDA;
    if (na == 0 || nb == 0) return BSH_OK;
    if (!work || work_bytes < bsh_coincidence_workspace(na, nb)) return BSH_ERR_WORKSPACE;
    unsigned char* w = static_cast<unsigned char*>(work);
    double* ra = reinterpret_cast<double*>(w);
    double* rb = reinterpret_cast<double*>(w + al256((size_t)na * 48));
    const PostConst c = make_const(*pp, pp->d_coinc);
    res_kernel<<<blocks_for(na), 256, 0, st>>>(pa, na, c, ra);
    res_kernel<<<blocks_for(nb), 256, 0, st>>>(pb, nb, c, rb);
    const dim3 grid((unsigned)((nb + TB - 1) / TB), (unsigned)((na + TB - 1) / TB));
    coinc_kernel<<<grid, TB, 0, st>>>(pa, ra, sa, va, na, pb, rb, sb, vb, nb, c, pairs, centroid, sig, cap, n_pairs);
    return cudaGetLastError() == cudaSuccess ? BSH_OK : BSH_ERR_CUDA;
}
