// Toplist merge (Sec. IV.C): each region (sky patch of a problem) collects the
// per-CTA candidate lists written by the number-count kernel, keeps the
// top_k largest keys (s_H, ties by smaller template id) and writes them sorted.
#include "bsh_internal.cuh"
#include "select.cuh"

namespace bsh {
namespace {

constexpr int MT = 512;

__global__ void __launch_bounds__(MT) merge_kernel(const MergeArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ SelectSmem sm;
    __shared__ int s_n;
    const int r = blockIdx.x;
    const int v0 = a.region_visit_off[r], v1 = a.region_visit_off[r + 1];
    const int nseg = v1 - v0;
    auto seg = [&](int sg, const Entry*& base, int& cnt) {
        const int v = a.region_visits[v0 + sg];
        base = a.visit_buf + (size_t)v * a.cap;
        cnt = a.visit_count[v];
    };
    int total = 0;
    for (int sg = 0; sg < nseg; ++sg) {
        const Entry* bp;
        int c;
        seg(sg, bp, c);
        total += c;
    }
    const int k = a.top_k;
    unsigned long long tau = 0ull;
    if (total > k) tau = cta_kth_largest<MT>(nseg, seg, k, sm);
    const int n = total < k ? total : k;
    // gather the survivors (unordered) into the region's scratch
    Entry* scr = a.scratch + (size_t)r * k;
    if (threadIdx.x == 0) s_n = 0;
    __syncthreads();
    for (int sg = 0; sg < nseg; ++sg) {
        const Entry* bp;
        int c;
        seg(sg, bp, c);
        for (int e = threadIdx.x; e < c; e += MT) {
            const Entry x = bp[e];
            if (x.key >= tau) {
                const int p = atomicAdd(&s_n, 1);
                if (p < k) scr[p] = x;
            }
        }
    }
    __syncthreads();
    // sort by key, descending
    int n2 = 1;
    while (n2 < n) n2 <<= 1;
    unsigned long long* key = reinterpret_cast<unsigned long long*>(smem);
    int* idx = reinterpret_cast<int*>(smem + (size_t)n2 * 8);
    for (int e = threadIdx.x; e < n2; e += MT) {
        key[e] = e < n ? scr[e].key : 0ull;
        idx[e] = e;
    }
    cta_bitonic_desc<MT>(key, idx, n2);
    const int q = a.region_problem[r];
    const ProbDev& P = a.probs[q];
    const int patch = r - P.region_base;
    const long long gbase = P.patch_start[patch] * (long long)P.B * P.n_f0;
    bsh_cand* out = a.out + (size_t)r * k;
    for (int e = threadIdx.x; e < n; e += MT) {
        const Entry x = scr[idx[e]];
        bsh_cand c;
        const uint32_t lid = 0xffffffffu - (uint32_t)(x.key & 0xffffffffull);
        c.template_id = gbase + (long long)lid;
        c.s_h = order_float((uint32_t)(x.key >> 32));
        c.n_w = x.n_w;
        c.n_unw = x.n_unw;
        c.power = 0.f;
        c.s_p = 0.f;
        c.region = r;
        out[e] = c;
    }
    if (threadIdx.x == 0) {
        a.n_out[r] = n;
        if (s_n != n) set_status(a.status, ST_ARG);
    }
}

}  // namespace

void launch_merge(const MergeArgs& a, int regions, cudaStream_t st) {
    if (regions <= 0) return;
    int n2 = 1;
    while (n2 < a.top_k) n2 <<= 1;
    const int smem = n2 * 12;
    static int s_merge = 0;
    ensure_smem(merge_kernel, smem, &s_merge);
    merge_kernel<<<regions, MT, smem, st>>>(a);
}

}  // namespace bsh
