// Peakgram (Sec. IV.A, Eq. (20)-(21)): normalised power rho = P / <n>^2 with
// <n>^2 = (running median over `window` bins) / ln 2, and the bit-packed
// 1/0 map rho > rho_th.  With window == 0 the input already is rho.
#include "bsh_internal.cuh"

namespace bsh {
namespace {

constexpr double kLn2 = 0.69314718055994530942;

// window == 0: one warp per 32-bin word; the ballot forms the word.
__global__ void peakgram_direct(const float* __restrict__ P, int N, int K, double rho_th,
                                float* __restrict__ rho, uint32_t* __restrict__ bits, int W) {
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (gw >= (long long)N * W) return;                // warp-uniform
    const int i = (int)(gw / W), wd = (int)(gw % W);
    const int k = wd * 32 + lane;
    float x = 0.f;
    if (k < K) x = P[(size_t)i * K + k];
    const bool on = (k < K) && ((double)x > rho_th);
    const unsigned m = __ballot_sync(0xffffffffu, on);
    if (rho && k < K) rho[(size_t)i * K + k] = x;
    if (lane == 0) bits[(size_t)i * W + wd] = m;
}

// Running median: one CTA per SFT row, the row staged in shared memory.  The median of a
// window is its element of rank half = window / 2 (0-based, ascending): the value x with
// #(y < x) <= half < #(y <= x).
//
// Each thread takes a segment of kSeg consecutive bins.  It finds the first bin's median by
// rank selection, then slides the window one bin at a time.  A slide removes one element and
// adds one, so x's counts #(y < x) and #(y <= x) change by at most one each and the new median
// is x itself, its successor min{y > x} or its predecessor max{y < x} in the new window: the
// counts are updated from the two elements in O(1), and only a move of the median takes one
// pass over the window (the new median's multiplicity comes from the same pass).  kSeg is odd,
// so the segments' windows start in distinct banks and the lanes of a warp never conflict.
constexpr int kSeg = 63;

// Median of w[0, window) by rank selection; *less, *leq: its counts in the window.
__device__ float median_select(const float* w, int window, int half, int* less, int* leq) {
    for (int q = 0; q < window; ++q) {
        const float x = w[q];
        int lt = 0, le = 0;
        for (int r = 0; r < window; ++r) {
            const float y = w[r];
            lt += (y < x);
            le += (y <= x);
        }
        if (lt <= half && le > half) {
            *less = lt;
            *leq = le;
            return x;
        }
    }
    *less = 0;   // unreachable for finite inputs: some element always holds the middle rank
    *leq = window;
    return w[0];
}

__global__ void peakgram_median(const float* __restrict__ P, int N, int K, int window, double rho_th,
                                float* __restrict__ rho, uint32_t* __restrict__ bits, int W) {
    extern __shared__ float s_row[];
    uint32_t* s_bits = reinterpret_cast<uint32_t*>(s_row + K);   // [W] this row's peakgram words
    const int i = blockIdx.x;
    const float* row = P + (size_t)i * K;
    for (int k = threadIdx.x; k < K; k += blockDim.x) s_row[k] = row[k];
    for (int wd = threadIdx.x; wd < W; wd += blockDim.x) s_bits[wd] = 0u;
    __syncthreads();
    const int half = window / 2;
    const int a_max = K - window;
    const int nseg = (K + kSeg - 1) / kSeg;
    for (int seg = threadIdx.x; seg < nseg; seg += blockDim.x) {
        const int k0 = seg * kSeg;
        const int k1 = min(k0 + kSeg, K);
        int a = min(max(k0 - half, 0), a_max);
        int less, leq;
        float m = median_select(s_row + a, window, half, &less, &leq);
        for (int k = k0; k < k1; ++k) {
            const int an = min(max(k - half, 0), a_max);
            if (an != a) {   // the window moved up by one bin
                const float xo = s_row[a], xi = s_row[a + window];
                less += (int)(xi < m) - (int)(xo < m);
                leq += (int)(xi <= m) - (int)(xo <= m);
                a = an;
                if (leq <= half) {          // the median moved up to m's successor
                    float nx = m;
                    int c = 0;
                    for (int r = 0; r < window; ++r) {
                        const float y = s_row[a + r];
                        if (y > m) {
                            if (c == 0 || y < nx) {
                                nx = y;
                                c = 1;
                            } else if (y == nx) {
                                ++c;
                            }
                        }
                    }
                    less = leq;
                    leq += c;
                    m = nx;
                } else if (less > half) {   // down to m's predecessor
                    float nx = m;
                    int c = 0;
                    for (int r = 0; r < window; ++r) {
                        const float y = s_row[a + r];
                        if (y < m) {
                            if (c == 0 || y > nx) {
                                nx = y;
                                c = 1;
                            } else if (y == nx) {
                                ++c;
                            }
                        }
                    }
                    leq = less;
                    less -= c;
                    m = nx;
                }
            }
            const double md = (double)m;
            const double lhs = __dmul_rn((double)s_row[k], kLn2);
            const double rhs = __dmul_rn(rho_th, md);
            if (lhs > rhs) atomicOr(&s_bits[k >> 5], 1u << (k & 31));
            if (rho) rho[(size_t)i * K + k] = __double2float_rn(__ddiv_rn(lhs, md));
        }
    }
    __syncthreads();
    for (int wd = threadIdx.x; wd < W; wd += blockDim.x) bits[(size_t)i * W + wd] = s_bits[wd];
}

}  // namespace

void launch_peakgram(const float* power, int N, int K, int window, double rho_th, float* rho,
                     uint32_t* bits, int W, cudaStream_t st) {
    if (N <= 0) return;
    if (window == 0) {
        const long long warps = (long long)N * W;
        const int threads = 256;
        const long long blocks = (warps * 32 + threads - 1) / threads;
        peakgram_direct<<<(unsigned)blocks, threads, 0, st>>>(power, N, K, rho_th, rho, bits, W);
    } else {
        const int threads = 128;
        const int bytes = (K + W) * (int)sizeof(float);
        static int s_med = 0;
        ensure_smem(peakgram_median, bytes, &s_med);
        peakgram_median<<<N, threads, (size_t)bytes, st>>>(power, N, K, window, rho_th, rho, bits, W);
    }
}

}  // namespace bsh
