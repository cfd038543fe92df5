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

// Running median: one CTA per SFT row, the row staged in shared memory.  The
// median of the shifted window is the element whose rank brackets the middle:
// #less <= half < #less_or_equal.
__global__ void peakgram_median(const float* __restrict__ P, int N, int K, int window, double rho_th,
                                float* __restrict__ rho, uint32_t* __restrict__ bits, int W) {
    extern __shared__ float s_row[];
    const int i = blockIdx.x;
    const float* row = P + (size_t)i * K;
    for (int k = threadIdx.x; k < K; k += blockDim.x) s_row[k] = row[k];
    __syncthreads();
    const int half = window / 2;
    const int kend = W * 32;
    for (int k0 = 0; k0 < kend; k0 += blockDim.x) {
        const int k = k0 + threadIdx.x;
        bool on = false;
        if (k < K) {
            int a = k - half;
            a = a < 0 ? 0 : a;
            a = (a + window > K) ? K - window : a;
            float m = s_row[a];
            for (int q = 0; q < window; ++q) {
                const float x = s_row[a + q];
                int less = 0, leq = 0;
                for (int r = 0; r < window; ++r) {
                    const float y = s_row[a + r];
                    less += (y < x);
                    leq += (y <= x);
                }
                if (less <= half && leq > half) { m = x; break; }
            }
            const double md = (double)m;
            const double lhs = __dmul_rn((double)s_row[k], kLn2);
            const double rhs = __dmul_rn(rho_th, md);
            on = lhs > rhs;
            if (rho) rho[(size_t)i * K + k] = __double2float_rn(__ddiv_rn(lhs, md));
        }
        const unsigned mk = __ballot_sync(0xffffffffu, on);
        if ((threadIdx.x & 31) == 0 && k < kend) bits[(size_t)i * W + (k >> 5)] = mk;
    }
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
        static int s_med = 0;
        ensure_smem(peakgram_median, K * (int)sizeof(float), &s_med);
        peakgram_median<<<N, threads, (size_t)K * sizeof(float), st>>>(power, N, K, window, rho_th, rho,
                                                                       bits, W);
    }
}

}  // namespace bsh
