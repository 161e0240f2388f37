// sgf_fft.cuh -- block-wide complex FFT in shared memory (device code only).
//
// The paper computes its convolutions with "the fast Fourier transform"
// (Sec. 2.2) without naming a scheme; this engine is a Stockham autosort
// transform (natural order in, natural order out) with radix-4 stages and
// one radix-2 stage when log2(N) is odd.  All threads of the block cooperate;
// each stage stages its butterflies' inputs in registers, synchronises, and
// writes the outputs back to the same buffer, so one N-point buffer per
// sequence suffices.  B sequences of length N lie back to back in `buf`.
//
// Twiddles come from a table of W_P^k = exp(-2 pi i k / P), P = 2N, built on
// the host from extended-precision sines and cosines (W_N^q = W_P^{2q}).
// The forward transform uses exp(-i...), the inverse exp(+i...), neither scaled.
#pragma once
#include <cuda_runtime.h>

namespace sgf {

template <typename C> struct Real;
template <> struct Real<float2> { using T = float; };
template <> struct Real<double2> { using T = double; };

template <typename C>
__device__ __forceinline__ C mk(typename Real<C>::T x, typename Real<C>::T y) { C c; c.x = x; c.y = y; return c; }
template <typename C>
__device__ __forceinline__ C cadd(C a, C b) { return mk<C>(a.x + b.x, a.y + b.y); }
template <typename C>
__device__ __forceinline__ C csub(C a, C b) { return mk<C>(a.x - b.x, a.y - b.y); }
template <typename C>
__device__ __forceinline__ C cmul(C a, C b) { return mk<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
// a * conj(b)
template <typename C>
__device__ __forceinline__ C cmulc(C a, C b) { return mk<C>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y); }
template <typename C>
__device__ __forceinline__ C cconj(C a) { return mk<C>(a.x, -a.y); }
template <typename C>
__device__ __forceinline__ C cscale(C a, typename Real<C>::T s) { return mk<C>(a.x * s, a.y * s); }
// multiply by -i (forward) or +i (inverse)
template <typename C, bool INV>
__device__ __forceinline__ C rot(C a) { return INV ? mk<C>(-a.y, a.x) : mk<C>(a.y, -a.x); }

template <typename C>
__device__ __forceinline__ C ldg_c(const C *p) { return __ldg(p); }

// Maximum complex values a thread holds per stage: B * N / blockDim.x <= kFftVpt.
constexpr int kFftVpt = 16;

template <typename C, bool INV>
__device__ __forceinline__ void radix4(C &v0, C &v1, C &v2, C &v3)
{
    C a0 = cadd(v0, v2), a1 = csub(v0, v2), a2 = cadd(v1, v3), a3 = rot<C, INV>(csub(v1, v3));
    v0 = cadd(a0, a2);
    v1 = cadd(a1, a3);
    v2 = csub(a0, a2);
    v3 = csub(a1, a3);
}

// In-place block FFT of B sequences of length N = 2^logN in shared memory.
// tw: W_P^k table in global memory, P = 2N.  Ends with a __syncthreads().
template <typename C, bool INV>
__device__ void block_fft(C *buf, int N, int logN, int B, const C *tw)
{
    const int nt = blockDim.x, tid = threadIdx.x;
    int Ns = 1;
    // radix-4 stages
    for (int st = 0; st < (logN >> 1); ++st) {
        const int q = N >> 2;            // butterflies per sequence
        const int nb = B * q;
        C v[kFftVpt / 4][4];
#pragma unroll
        for (int it = 0; it < kFftVpt / 4; ++it) {
            const int b = tid + it * nt;
            if (b < nb) {
                const int seq = b / q, j = b - seq * q;
                const C *in = buf + (size_t)seq * N + j;
#pragma unroll
                for (int r = 0; r < 4; ++r)
                    v[it][r] = in[r * q];
            }
        }
        __syncthreads();
        const int tstride = (2 * N) / (Ns * 4);  // W_{4 Ns} = W_P^{tstride}
#pragma unroll
        for (int it = 0; it < kFftVpt / 4; ++it) {
            const int b = tid + it * nt;
            if (b < nb) {
                const int seq = b / q, j = b - seq * q;
                const int k = j & (Ns - 1);
                if (Ns > 1) {
#pragma unroll
                    for (int r = 1; r < 4; ++r) {
                        const C w = ldg_c(tw + r * k * tstride);
                        v[it][r] = INV ? cmulc(v[it][r], w) : cmul(v[it][r], w);
                    }
                }
                radix4<C, INV>(v[it][0], v[it][1], v[it][2], v[it][3]);
                C *out = buf + (size_t)seq * N + (j - k) * 4 + k;
#pragma unroll
                for (int r = 0; r < 4; ++r)
                    out[r * Ns] = v[it][r];
            }
        }
        __syncthreads();
        Ns <<= 2;
    }
    // final radix-2 stage when log2(N) is odd
    if (Ns < N) {
        const int q = N >> 1;
        const int nb = B * q;
        C v[kFftVpt / 2][2];
#pragma unroll
        for (int it = 0; it < kFftVpt / 2; ++it) {
            const int b = tid + it * nt;
            if (b < nb) {
                const int seq = b / q, j = b - seq * q;
                const C *in = buf + (size_t)seq * N + j;
                v[it][0] = in[0];
                v[it][1] = in[q];
            }
        }
        __syncthreads();
        const int tstride = (2 * N) / (Ns * 2);
#pragma unroll
        for (int it = 0; it < kFftVpt / 2; ++it) {
            const int b = tid + it * nt;
            if (b < nb) {
                const int seq = b / q, j = b - seq * q;
                const int k = j & (Ns - 1);
                if (Ns > 1) {
                    const C w = ldg_c(tw + k * tstride);
                    v[it][1] = INV ? cmulc(v[it][1], w) : cmul(v[it][1], w);
                }
                const C a = v[it][0], b2 = v[it][1];
                C *out = buf + (size_t)seq * N + (j - k) * 2 + k;
                out[0] = cadd(a, b2);
                out[Ns] = csub(a, b2);
            }
        }
        __syncthreads();
    }
}

}  // namespace sgf
