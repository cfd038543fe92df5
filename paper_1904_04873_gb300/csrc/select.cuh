// CTA-wide selection helpers for the toplists (Sec. IV.C): exact k-th largest
// 64-bit key by MSB-first radix selection, stable in-place compaction, and a
// bitonic sort of (key, index) pairs in shared memory.  Keys are unique
// (they embed the template id), so "the k largest keys" is one set.
#pragma once

#include "bsh_internal.cuh"

namespace bsh {

struct SelectSmem {
    unsigned hist[256];
    unsigned long long prefix;
    int rem;
    int warp_tot[33];
    int total;
};

// Segments: keys of seg s are at base[s] (Entry stride), count n[s].  Returns
// the k-th largest key over all segments (1 <= k <= total).
template <int THREADS, class SegFn>
__device__ unsigned long long cta_kth_largest(int nseg, SegFn seg, int k, SelectSmem& sm) {
    unsigned long long prefix = 0ull, pmask = 0ull;
    int rem = k;
    for (int shift = 56; shift >= 0; shift -= 8) {
        for (int b = threadIdx.x; b < 256; b += THREADS) sm.hist[b] = 0u;
        __syncthreads();
        for (int sg = 0; sg < nseg; ++sg) {
            const Entry* base;
            int n;
            seg(sg, base, n);
            for (int e = threadIdx.x; e < n; e += THREADS) {
                const unsigned long long key = base[e].key;
                if ((key & pmask) == prefix) atomicAdd(&sm.hist[(unsigned)(key >> shift) & 255u], 1u);
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int c = 0, b = 255;
            for (; b > 0; --b) {
                if (c + (int)sm.hist[b] >= rem) break;
                c += (int)sm.hist[b];
            }
            sm.rem = rem - c;
            sm.prefix = prefix | ((unsigned long long)b << shift);
        }
        __syncthreads();
        prefix = sm.prefix;
        rem = sm.rem;
        pmask |= 255ull << shift;
        __syncthreads();
    }
    return prefix;
}

// Stable in-place compaction of arr[0..n) keeping keys >= tau; returns the new count.
template <int THREADS>
__device__ int cta_compact_ge(Entry* arr, int n, unsigned long long tau, SelectSmem& sm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int NW = THREADS / 32;
    int out = 0;
    for (int base = 0; base < n; base += THREADS) {
        const int e = base + threadIdx.x;
        Entry x;
        bool keep = false;
        if (e < n) {
            x = arr[e];
            keep = x.key >= tau;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, keep);
        if (lane == 0) sm.warp_tot[warp] = __popc(bal);
        __syncthreads();
        if (threadIdx.x == 0) {
            int acc = 0;
            for (int w = 0; w < NW; ++w) {
                const int t = sm.warp_tot[w];
                sm.warp_tot[w] = acc;
                acc += t;
            }
            sm.total = acc;
        }
        __syncthreads();
        if (keep) arr[out + sm.warp_tot[warp] + __popc(bal & ((1u << lane) - 1u))] = x;
        out += sm.total;
        __syncthreads();
    }
    return out;
}

// Sorts key[0..n2) (n2 a power of two) in descending order together with idx.
template <int THREADS>
__device__ void cta_bitonic_desc(unsigned long long* key, int* idx, int n2) {
    for (int size = 2; size <= n2; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            __syncthreads();
            for (int t = threadIdx.x; t < (n2 >> 1); t += THREADS) {
                const int lo = 2 * t - (t & (stride - 1));
                const int hi = lo + stride;
                const bool desc = (lo & size) == 0;
                const unsigned long long a = key[lo], b = key[hi];
                const bool swap = desc ? (a < b) : (a > b);
                if (swap) {
                    key[lo] = b;
                    key[hi] = a;
                    const int ti = idx[lo];
                    idx[lo] = idx[hi];
                    idx[hi] = ti;
                }
            }
        }
    }
    __syncthreads();
}

}  // namespace bsh
