// sgf_fft16.cuh -- register-resident block FFT (radix 16) for N in [16, 4096].
//
// Layout.  A CTA transforms B sequences of length N.  The data are cut into
// "slots" of 16 complex values: slot (s, j), j in [0, N/16), holds elements
// j + u*N/16 (u = 0..15) of sequence s, in one thread's registers.  Every
// stage of the Stockham autosort recursion reads its butterfly inputs in
// exactly this pattern; radix-16 stages run while 16 divides the remaining
// length and one radix-2/4/8 stage closes (a slot then holds 16/R
// butterflies).  Between stages the data go through shared memory once
// (padded by one element every 16 so strided writes do not collide in banks).
// The last stage's outputs land in the same slot pattern, in natural order:
// after a forward transform, slot (s, j) holds bins j + u*N/16.  So data can be
// loaded from global memory straight into registers, transformed, multiplied
// bin by bin, inverse-transformed and stored, with the shared-memory traffic
// limited to the exchanges between stages.
//
// Twiddles: every stage after the first multiplies by W_{R Ns}^{r k}
// (k = the butterfly's index modulo Ns).  They come from per-stage tables laid
// out [r-1][k] (r = 1..R-1, k < Ns), so the threads of a warp, whose k are
// consecutive, read consecutive words (no bank conflicts); the tables are
// built on the host in extended precision and kept in shared memory.
// The in-register 16- and 8-point DFTs use the exact constants cos(pi/8),
// sin(pi/8) and sqrt(1/2).
#pragma once
#include <cstring>
#include "sgf_fft.cuh"
#ifdef __CUDACC__
#include "sgf_tc.cuh"
#endif

namespace sgf {

#define SGF_HD __host__ __device__ __forceinline__

template <typename C> struct K16;
template <> struct K16<float2> {
    static SGF_HD float c1() { return 0.92387953251128674f; }   // cos(pi/8)
    static SGF_HD float s1() { return 0.38268343236508978f; }   // sin(pi/8)
    static SGF_HD float h() { return 0.70710678118654752f; }    // sqrt(1/2)
};
template <> struct K16<double2> {
    static SGF_HD double c1() { return 0.92387953251128674; }
    static SGF_HD double s1() { return 0.38268343236508978; }
    static SGF_HD double h() { return 0.70710678118654752; }
};

template <typename C> SGF_HD C hmk(typename Real<C>::T x, typename Real<C>::T y) { C c; c.x = x; c.y = y; return c; }
template <typename C> SGF_HD C hadd(C a, C b) { return hmk<C>(a.x + b.x, a.y + b.y); }
template <typename C> SGF_HD C hsub(C a, C b) { return hmk<C>(a.x - b.x, a.y - b.y); }
template <typename C> SGF_HD C hmul(C a, C b) { return hmk<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
template <typename C> SGF_HD C hmulc(C a, C b) { return hmk<C>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y); }
// times exp(-i pi/2) (forward) / exp(+i pi/2) (inverse)
template <typename C, bool INV> SGF_HD C hrot(C a) { return INV ? hmk<C>(-a.y, a.x) : hmk<C>(a.y, -a.x); }

// Complex add and subtract of the butterflies.  For float2 on the device each is
// one packed two-lane FP32 instruction (add.rn.f32x2 / sub.rn.f32x2, sm_100 and
// later), the same two IEEE operations as the scalar form.
template <typename C> SGF_HD C badd(C a, C b) { return hadd(a, b); }
template <typename C> SGF_HD C bsub(C a, C b) { return hsub(a, b); }
template <>
SGF_HD float2 badd<float2>(float2 a, float2 b)
{
#if defined(__CUDA_ARCH__)
    unsigned long long ra, rb, rr;
    memcpy(&ra, &a, 8);
    memcpy(&rb, &b, 8);
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(rr) : "l"(ra), "l"(rb));
    float2 r;
    memcpy(&r, &rr, 8);
    return r;
#else
    return hadd(a, b);
#endif
}
template <>
SGF_HD float2 bsub<float2>(float2 a, float2 b)
{
#if defined(__CUDA_ARCH__)
    unsigned long long ra, rb, rr;
    memcpy(&ra, &a, 8);
    memcpy(&rb, &b, 8);
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(rr) : "l"(ra), "l"(rb));
    float2 r;
    memcpy(&r, &rr, 8);
    return r;
#else
    return hsub(a, b);
#endif
}

// 4-point DFT; the outputs 1 and 3 take the rotated difference (times -i
// forward, +i inverse) with scalar adds.
template <typename C, bool INV>
SGF_HD void hdft4(C &v0, C &v1, C &v2, C &v3)
{
    const C a0 = badd(v0, v2), a1 = bsub(v0, v2), a2 = badd(v1, v3), d = bsub(v1, v3);
    v0 = badd(a0, a2);
    v2 = bsub(a0, a2);
    if (INV) {
        v1 = hmk<C>(a1.x - d.y, a1.y + d.x);
        v3 = hmk<C>(a1.x + d.y, a1.y - d.x);
    } else {
        v1 = hmk<C>(a1.x + d.y, a1.y - d.x);
        v3 = hmk<C>(a1.x - d.y, a1.y + d.x);
    }
}

// multiply by W16^e (forward: exp(-2 pi i e/16)), e in 0..9
template <typename C, bool INV>
SGF_HD C w16(C a, int e)
{
    using T = typename Real<C>::T;
    const T c1 = K16<C>::c1(), s1 = K16<C>::s1(), h = K16<C>::h();
    T wr, wi;
    switch (e) {
    case 0: return a;
    case 1: wr = c1; wi = -s1; break;
    case 2: wr = h; wi = -h; break;
    case 3: wr = s1; wi = -c1; break;
    case 4: return hrot<C, INV>(a);
    case 6: wr = -h; wi = -h; break;
    case 9: wr = -c1; wi = s1; break;
    default: wr = 1; wi = 0; break;  // not used
    }
    if (INV)
        wi = -wi;
    return hmk<C>(a.x * wr - a.y * wi, a.x * wi + a.y * wr);
}

// In-place 16-point DFT in natural order: v[k] <- sum_n v[n] W16^{nk}.
template <typename C, bool INV>
SGF_HD void hdft16(C *v)
{
    C a[16];
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) {
        C x0 = v[n2], x1 = v[n2 + 4], x2 = v[n2 + 8], x3 = v[n2 + 12];
        hdft4<C, INV>(x0, x1, x2, x3);
        a[4 * n2 + 0] = x0;
        a[4 * n2 + 1] = w16<C, INV>(x1, n2);
        a[4 * n2 + 2] = w16<C, INV>(x2, 2 * n2);
        a[4 * n2 + 3] = w16<C, INV>(x3, 3 * n2);
    }
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
        C b0 = a[k1], b1 = a[4 + k1], b2 = a[8 + k1], b3 = a[12 + k1];
        hdft4<C, INV>(b0, b1, b2, b3);
        v[k1] = b0;
        v[k1 + 4] = b1;
        v[k1 + 8] = b2;
        v[k1 + 12] = b3;
    }
}

// W_{R Ns}^{r k} of stage table `tws` (see Fft16Plan).
template <typename C>
SGF_HD C stage_twiddle(const C *tws, int R, int Ns, int r, int k)
{
    if (Ns < 256)
        return tws[(r - 1) * Ns + k];
    const C a = tws[(r - 1) * 16 + (k & 15)];
    const C b = tws[(R - 1) * 16 + (r - 1) * (Ns >> 4) + (k >> 4)];
    return hmul(a, b);
}

// In-place R-point DFT (R = 2, 4, 8) of the values v[Q + r*(16/R)], r = 0..R-1;
// R and Q are compile-time so the register array is never indexed at run time.
template <typename C, bool INV, int R, int Q>
SGF_HD void hdft_small(C *v)
{
    constexpr int S = 16 / R;
    if (R == 2) {
        C a = v[Q], b = v[Q + S];
        v[Q] = badd(a, b);
        v[Q + S] = bsub(a, b);
    } else if (R == 4) {
        hdft4<C, INV>(v[Q], v[Q + S], v[Q + 2 * S], v[Q + 3 * S]);
    } else {  // R == 8: n = 2 n1 + n2, k = k1 + 4 k2
        C e0 = v[Q], e1 = v[Q + 2 * S], e2 = v[Q + 4 * S], e3 = v[Q + 6 * S];
        C o0 = v[Q + S], o1 = v[Q + 3 * S], o2 = v[Q + 5 * S], o3 = v[Q + 7 * S];
        hdft4<C, INV>(e0, e1, e2, e3);
        hdft4<C, INV>(o0, o1, o2, o3);
        o1 = w16<C, INV>(o1, 2);  // W8^1 = W16^2
        o2 = w16<C, INV>(o2, 4);  // W8^2
        o3 = w16<C, INV>(o3, 6);  // W8^3
        v[Q] = badd(e0, o0);
        v[Q + S] = badd(e1, o1);
        v[Q + 2 * S] = badd(e2, o2);
        v[Q + 3 * S] = badd(e3, o3);
        v[Q + 4 * S] = bsub(e0, o0);
        v[Q + 5 * S] = bsub(e1, o1);
        v[Q + 6 * S] = bsub(e2, o2);
        v[Q + 7 * S] = bsub(e3, o3);
    }
}

// The closing radix-R stage on one slot: 16/R butterflies, butterfly Q holding
// v[Q + r*(16/R)]; its twiddles are W_{R Ns}^{r k}.
template <typename C, bool INV, int R, int Q>
SGF_HD void stage_small_one(C *v, int N, int Ns, int j, const C *tw)
{
    constexpr int S = 16 / R;
    const int jq = j + Q * (N / 16);
    const int k = jq & (Ns - 1);
    if (Ns > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) {
            const C w = stage_twiddle(tw, R, Ns, r, k);  // this stage's table
            v[Q + r * S] = INV ? hmulc(v[Q + r * S], w) : hmul(v[Q + r * S], w);
        }
    }
    hdft_small<C, INV, R, Q>(v);
}

template <typename C, bool INV, int R>
SGF_HD void stage_small(C *v, int N, int Ns, int j, const C *tw)
{
    stage_small_one<C, INV, R, 0>(v, N, Ns, j, tw);
    if (16 / R > 1) stage_small_one<C, INV, R, (16 / R > 1 ? 1 : 0)>(v, N, Ns, j, tw);
    if (16 / R > 2) {
        stage_small_one<C, INV, R, (16 / R > 2 ? 2 : 0)>(v, N, Ns, j, tw);
        stage_small_one<C, INV, R, (16 / R > 3 ? 3 : 0)>(v, N, Ns, j, tw);
    }
    if (16 / R > 4) {
        stage_small_one<C, INV, R, (16 / R > 4 ? 4 : 0)>(v, N, Ns, j, tw);
        stage_small_one<C, INV, R, (16 / R > 5 ? 5 : 0)>(v, N, Ns, j, tw);
        stage_small_one<C, INV, R, (16 / R > 6 ? 6 : 0)>(v, N, Ns, j, tw);
        stage_small_one<C, INV, R, (16 / R > 7 ? 7 : 0)>(v, N, Ns, j, tw);
    }
}

SGF_HD int pad16(int i) { return i + (i >> 4); }

// Stage bookkeeping shared by the device engine, the host table builder and
// the host test emulator.  Stage st (> 0) multiplies by W_{R Ns}^{r k},
// r = 1..R-1, k < Ns.  For Ns < 256 its table is D[r-1][k] (at twoff[st]);
// for Ns >= 256 the twiddle is factored over k = 16 kh + kl into
// A[r-1][kl] = W_{R Ns}^{r kl} (16 per r) times B[r-1][kh] = W_{R Ns}^{16 r kh}
// (Ns/16 per r), which keeps the tables a few KB.  Within a warp kl runs
// over 16 consecutive values and kh over at most two, so the reads are
// conflict-free or broadcasts.
struct Fft16Plan {
    int N, logN, nst, S16, rlast;
    int twoff[5];
    int twlen;  // entries of all stage tables together
    SGF_HD void init(int n, int logn)
    {
        N = n;
        logN = logn;
        S16 = logn >> 2;
        rlast = 1 << (logn & 3);
        nst = S16 + (rlast > 1 ? 1 : 0);
        int off = 0, Ns = 1;
        for (int st = 0; st < 5; ++st) {
            twoff[st] = off;
            if (st < nst) {
                const int R = radix(st);
                if (st > 0)
                    off += Ns >= 256 ? (R - 1) * (16 + Ns / 16) : (R - 1) * Ns;
                Ns *= R;
            }
        }
        twlen = off;
    }
    SGF_HD int radix(int st) const { return st < S16 ? 16 : rlast; }
};

// One stage's arithmetic on a slot: twiddles + DFT.  Ns = product of earlier radices.
template <typename C, bool INV>
SGF_HD void fft16_stage_compute(C *v, const Fft16Plan &pl, int st, int Ns, int j, const C *tw)
{
    const int R = pl.radix(st), N = pl.N;
    const C *tws = tw + pl.twoff[st];  // [r-1][k], k < Ns
    if (R == 16) {
        const int k = j & (Ns - 1);
        if (Ns > 1) {
#pragma unroll
            for (int r = 1; r < 16; ++r) {
                const C w = stage_twiddle(tws, 16, Ns, r, k);
                v[r] = INV ? hmulc(v[r], w) : hmul(v[r], w);
            }
        }
        hdft16<C, INV>(v);
    } else if (R == 8) {
        stage_small<C, INV, 8>(v, N, Ns, j, tws);
    } else if (R == 4) {
        stage_small<C, INV, 4>(v, N, Ns, j, tws);
    } else {
        stage_small<C, INV, 2>(v, N, Ns, j, tws);
    }
}

// Where a non-final (radix-16) stage writes output r of slot j.
SGF_HD int fft16_out_index(int j, int Ns, int r)
{
    const int k = j & (Ns - 1);
    return (j - k) * 16 + k + r * Ns;
}

#ifdef __CUDACC__
// Block-wide transform of the slot held in v.  sbuf: shared memory, sequence s
// at s * SP (SP >= N + N/16); tw: the stage twiddle tables (shared memory).
// Every thread of the block must call this (active == false: a thread without
// a slot still takes part in the barriers).  sbuf is first
// written after a barrier, so it may still be in use on entry; the last stage
// reads sbuf without a closing barrier, so callers synchronise before reusing it.
template <typename C, bool INV>
__device__ __forceinline__ void fft16_block(C *v, C *sbuf, int s, int SP, int j, bool active,
                                            const Fft16Plan &pl, const C *tw)
{
    const int N = pl.N, Q = N >> 4;
    C *seq = sbuf + (size_t)s * SP;
    int Ns = 1;
    for (int st = 0; st < pl.nst; ++st) {
        if (st > 0) {
            __syncthreads();  // previous stage's stores are visible
            if (active) {
#pragma unroll
                for (int u = 0; u < 16; ++u)
                    v[u] = seq[pad16(j + u * Q)];
            }
        }
        if (active)
            fft16_stage_compute<C, INV>(v, pl, st, Ns, j, tw);
        if (st + 1 < pl.nst) {
            __syncthreads();  // every thread has read this stage's inputs
            if (active) {
#pragma unroll
                for (int r = 0; r < 16; ++r)
                    seq[pad16(fft16_out_index(j, Ns, r))] = v[r];
            }
        }
        Ns *= pl.radix(st);
    }
}
#endif


// ---------------------------------------------------------------------------
// Compile-time engine: the same transform with N a template constant, so every
// stride, radix, twiddle-table offset and padded index folds at compile time.
template <int LOGN>
struct F16 {
    static constexpr int N = 1 << LOGN;
    static constexpr int Q = N >> 4;
    static constexpr int S16 = LOGN >> 2;
    static constexpr int RL = 1 << (LOGN & 3);
    static constexpr int NST = S16 + (RL > 1 ? 1 : 0);
    static constexpr int radix(int st) { return st < S16 ? 16 : RL; }
    static constexpr int ns(int st)
    {
        int n = 1;
        for (int s = 0; s < st; ++s)
            n *= radix(s);
        return n;
    }
    static constexpr int tsize(int st)
    {
        return st == 0 ? 0 : (ns(st) >= 256 ? (radix(st) - 1) * (16 + ns(st) / 16) : (radix(st) - 1) * ns(st));
    }
    static constexpr int twoff(int st)
    {
        int o = 0;
        for (int s = 1; s < st; ++s)
            o += tsize(s);
        return o;
    }
    static constexpr int twlen = twoff(NST);
};

template <typename C, int R, int NS>
SGF_HD C stage_tw(const C *tws, int r, int k)
{
    if constexpr (NS < 256) {
        return tws[(r - 1) * NS + k];
    } else {
        const C a = tws[(r - 1) * 16 + (k & 15)];
        const C b = tws[(R - 1) * 16 + (r - 1) * (NS >> 4) + (k >> 4)];
        return hmul(a, b);
    }
}

template <typename C, bool INV, int N, int R, int NS, int QB>
SGF_HD void stage_small_ct(C *v, int j, const C *tws)
{
    if constexpr (QB < 16 / R) {
        constexpr int S = 16 / R;
        if constexpr (NS > 1) {
            const int k = (j + QB * (N / 16)) & (NS - 1);
#pragma unroll
            for (int r = 1; r < R; ++r) {
                const C w = stage_tw<C, R, NS>(tws, r, k);
                v[QB + r * S] = INV ? hmulc(v[QB + r * S], w) : hmul(v[QB + r * S], w);
            }
        }
        hdft_small<C, INV, R, QB>(v);
        stage_small_ct<C, INV, N, R, NS, QB + 1>(v, j, tws);
    }
}

// Twiddles of a radix-16 stage ST on one slot.
template <typename C, bool INV, int LOGN, int ST>
SGF_HD void stage_tw16(C *v, int j, const C *tw)
{
    using P = F16<LOGN>;
    constexpr int NS = P::ns(ST);
    if constexpr (NS > 1) {
        const C *tws = tw + P::twoff(ST);
        const int k = j & (NS - 1);
#pragma unroll
        for (int r = 1; r < 16; ++r) {
            const C w = stage_tw<C, 16, NS>(tws, r, k);
            v[r] = INV ? hmulc(v[r], w) : hmul(v[r], w);
        }
    }
}

// Arithmetic of stage ST on one slot.
template <typename C, bool INV, int LOGN, int ST>
SGF_HD void stage_ct(C *v, int j, const C *tw)
{
    using P = F16<LOGN>;
    constexpr int R = P::radix(ST), NS = P::ns(ST);
    if constexpr (R == 16) {
        stage_tw16<C, INV, LOGN, ST>(v, j, tw);
        hdft16<C, INV>(v);
    } else {
        stage_small_ct<C, INV, P::N, R, NS, 0>(v, j, tw + P::twoff(ST));
    }
}

#ifdef __CUDACC__
// Stages ST.. of the block transform (see fft16_block); B sequences per slot
// (B = 1 or 2: a thread may carry the same slot of two sequences, which then
// share the barriers), sequence b at sbuf + b * SP.  TC (float only): the
// Barrier of a transform's exchanges: the whole block (HB = 0), or, where the
// two parity halves of a block run independent transforms on disjoint exchange
// buffers, the named barrier 1 + half over the HB threads of that half (HB a
// multiple of 32, each half whole warps), so the halves need not wait for each
// other between stages.
// (half 2 and 3: the two halves of a second row pair in k_row_fwd_m2, named
// barriers 3 and 4; immediate ids keep the block's barrier count at 5)
template <int HB>
__device__ __forceinline__ void xsync(int half)
{
    if constexpr (HB == 0)
        __syncthreads();
    else if (half == 0)  // warp-uniform
        asm volatile("bar.sync 1, %0;" ::"n"(HB) : "memory");
    else if (half == 1)
        asm volatile("bar.sync 2, %0;" ::"n"(HB) : "memory");
    else if (half == 2)
        asm volatile("bar.sync 3, %0;" ::"n"(HB) : "memory");
    else
        asm volatile("bar.sync 4, %0;" ::"n"(HB) : "memory");
}

// 16-point DFTs of the radix-16 stages run as split-BF16 tensor-core tiles
// (sgf_tc.cuh, context tc); twiddles, exchanges and the closing radix-2/4/8
// stage stay in FP32.
template <typename C, bool INV, int LOGN, int B, int ST, bool TC = false, int HB = 0>
__device__ __forceinline__ void fft_stages(C (*v)[16], C *sbuf, int SP, int j, bool active, const C *tw,
                                           TcCtx *tc = nullptr, int half = 0)
{
    using P = F16<LOGN>;
    static_assert(HB == 0 || (!TC && HB % 32 == 0), "half barriers: FP32/FP64 engine, whole warps per half");
    if constexpr (ST < P::NST) {
        constexpr int Q = P::Q, NS = P::ns(ST);
        if constexpr (ST > 0) {
            xsync<HB>(half);  // previous stage's stores are visible
            if (active) {
#pragma unroll
                for (int bb = 0; bb < B; ++bb)
#pragma unroll
                    for (int u = 0; u < 16; ++u)
                        v[bb][u] = sbuf[bb * SP + pad16(j + u * Q)];
            }
        }
        if constexpr (TC && P::radix(ST) == 16) {
            if (active) {
#pragma unroll
                for (int bb = 0; bb < B; ++bb)
                    stage_tw16<C, INV, LOGN, ST>(v[bb], j, tw);
            }
            tc_dft16<INV, B>(v, *tc, active);
        } else if (active) {
#pragma unroll
            for (int bb = 0; bb < B; ++bb)
                stage_ct<C, INV, LOGN, ST>(v[bb], j, tw);
        }
        if constexpr (ST + 1 < P::NST) {
            xsync<HB>(half);  // every thread has read this stage's inputs
            if (active) {
                const int k = j & (NS - 1);
                const int base = (j - k) * 16 + k;
#pragma unroll
                for (int bb = 0; bb < B; ++bb)
#pragma unroll
                    for (int r = 0; r < 16; ++r)
                        sbuf[bb * SP + pad16(base + r * NS)] = v[bb][r];
            }
        }
        fft_stages<C, INV, LOGN, B, ST + 1, TC, HB>(v, sbuf, SP, j, active, tw, tc, half);
    }
}

// Block-wide transform, compile-time N: as fft16_block, for B slots per thread.
// HB > 0: the transform of one parity half (`half`) with that half's named
// barrier (xsync); the caller separates it from the other half's use of the
// same shared memory by block barriers before and after.
template <typename C, bool INV, int LOGN, int B = 1, bool TC = false, int HB = 0>
__device__ __forceinline__ void fft_ct(C (*v)[16], C *sbuf, int SP, int j, bool active, const C *tw,
                                       TcCtx *tc = nullptr, int half = 0)
{
    fft_stages<C, INV, LOGN, B, 0, TC, HB>(v, sbuf, SP, j, active, tw, tc, half);
}
#endif

// ---------------------------------------------------------------------------
// Register-twiddle engine.  A thread that keeps one slot j for the whole life
// of a kernel (a CTA walking many columns or row pairs) holds the twiddles of
// its slot in registers instead of reading shared tables at every stage:
// stage st >= 1 of radix R needs W_{R Ns}^{r k} for r = 1..R-1 with
// k = (j + QB N/16) mod Ns for each of its 16/R butterflies QB, at most 15
// values.  They are read once, at the start of the kernel, from the full table
// W_N^i (i < N, built on the host in extended precision): W_{R Ns}^{r k} =
// W_N^{r k N / (R Ns)}.
//
// Radix plans (the autotuner chooses): PLAN 0 runs radix-16 stages and closes
// with one radix-2/4/8 stage when 16 does not divide the length (the table
// engine's order); PLAN 1 puts that small stage first (n = 1024: 4.16.16,
// 2048: 8.16.16) or, for n = 4096, runs four radix-8 stages (8.8.8.8).  Every
// stage reads the slot pattern j + u N/16; a radix-R stage with R < 16 holds
// 16/R butterflies per slot and writes butterfly QB's outputs, like a radix-16
// stage writes its one butterfly's, at (jq - k) R + k + r Ns, jq = j + QB N/16.
template <int LOGN, int PLAN>
struct FR {
    static constexpr int N = 1 << LOGN;
    static constexpr int Q = N >> 4;
    static constexpr int S16 = LOGN >> 2;
    static constexpr int RL = 1 << (LOGN & 3);
    static constexpr bool EIGHTS = PLAN == 1 && (LOGN & 3) == 0 && LOGN % 3 == 0;  // 4096 = 8^4 (512 = 8^3)
    static constexpr int NST = EIGHTS ? LOGN / 3 : S16 + (RL > 1 ? 1 : 0);
    static constexpr int radix(int st)
    {
        return EIGHTS ? 8 : PLAN == 0 ? (st < S16 ? 16 : RL) : (RL > 1 && st == 0 ? RL : 16);
    }
    static constexpr int ns(int st)
    {
        int n = 1;
        for (int s = 0; s < st; ++s)
            n *= radix(s);
        return n;
    }
};

template <typename C, int LOGN, int PLAN, int ST>
__device__ __forceinline__ void load_stage_twiddles(C (&w)[15], const C *twn, int j)
{
    using P = FR<LOGN, PLAN>;
    constexpr int R = P::radix(ST), NS = P::ns(ST), S = 16 / R, N = P::N, STEP = N / (R * NS);
#pragma unroll
    for (int qb = 0; qb < S; ++qb) {
        const int k = (j + qb * P::Q) & (NS - 1);
#pragma unroll
        for (int r = 1; r < R; ++r)
            w[qb * (R - 1) + r - 1] = twn[(r * k * STEP) & (N - 1)];
    }
}

// Twiddles of every stage after the first: w[st - 1] for st = 1 .. NST - 1.
template <typename C, int LOGN, int PLAN, int ST = 1>
__device__ __forceinline__ void load_twiddles_rt(C (*w)[15], const C *twn, int j)
{
    if constexpr (ST < FR<LOGN, PLAN>::NST) {
        load_stage_twiddles<C, LOGN, PLAN, ST>(w[ST - 1], twn, j);
        load_twiddles_rt<C, LOGN, PLAN, ST + 1>(w, twn, j);
    }
}

template <typename C, bool INV, int R, int QB>
SGF_HD void stage_small_rt(C *v, const C *w)
{
    if constexpr (QB < 16 / R) {
        constexpr int S = 16 / R;
#pragma unroll
        for (int r = 1; r < R; ++r)
            v[QB + r * S] = INV ? hmulc(v[QB + r * S], w[QB * (R - 1) + r - 1]) : hmul(v[QB + r * S], w[QB * (R - 1) + r - 1]);
        hdft_small<C, INV, R, QB>(v);
        stage_small_rt<C, INV, R, QB + 1>(v, w);
    }
}

#ifdef __CUDACC__
// Barrier of a group of `count` threads (a multiple of 32) on named barrier `id`.
__device__ __forceinline__ void group_sync(unsigned id, unsigned count)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// fft_stages with the stage twiddles in registers (w, see load_twiddles_rt), a
// radix plan, and the exchanges of a group of threads on its own named barrier.
// B sequences per thread, sequence b at sbuf + b * SP; same entry and exit
// conditions as fft_stages (sbuf first written after a barrier, last stage read
// without a closing one).
template <typename C, bool INV, int LOGN, int PLAN, int B, int ST>
__device__ __forceinline__ void fft_stages_rt(C (*v)[16], C *sbuf, int SP, int j, const C (*w)[15], unsigned bar,
                                              unsigned count)
{
    using P = FR<LOGN, PLAN>;
    if constexpr (ST < P::NST) {
        constexpr int Q = P::Q, NS = P::ns(ST), R = P::radix(ST), S = 16 / R;
        if constexpr (ST > 0) {
            group_sync(bar, count);  // previous stage's stores are visible
#pragma unroll
            for (int bb = 0; bb < B; ++bb)
#pragma unroll
                for (int u = 0; u < 16; ++u)
                    v[bb][u] = sbuf[bb * SP + pad16(j + u * Q)];
        }
#pragma unroll
        for (int bb = 0; bb < B; ++bb) {
            if constexpr (R == 16) {
                if constexpr (ST > 0) {
#pragma unroll
                    for (int r = 1; r < 16; ++r)
                        v[bb][r] = INV ? hmulc(v[bb][r], w[ST - 1][r - 1]) : hmul(v[bb][r], w[ST - 1][r - 1]);
                }
                hdft16<C, INV>(v[bb]);
            } else if constexpr (ST > 0) {
                stage_small_rt<C, INV, R, 0>(v[bb], w[ST - 1]);
            } else {  // a first stage: no twiddles (Ns = 1)
                static_assert(NS == 1, "the first stage has Ns = 1");
                stage_small_ct<C, INV, P::N, R, 1, 0>(v[bb], j, static_cast<const C *>(nullptr));
            }
        }
        if constexpr (ST + 1 < P::NST) {
            group_sync(bar, count);  // every thread has read this stage's inputs
#pragma unroll
            for (int qb = 0; qb < S; ++qb) {
                const int jq = j + qb * Q;
                const int k = jq & (NS - 1);
                const int base = (jq - k) * R + k;
#pragma unroll
                for (int bb = 0; bb < B; ++bb)
#pragma unroll
                    for (int r = 0; r < R; ++r)
                        sbuf[bb * SP + pad16(base + r * NS)] = v[bb][qb + r * S];
            }
        }
        fft_stages_rt<C, INV, LOGN, PLAN, B, ST + 1>(v, sbuf, SP, j, w, bar, count);
    }
}
#endif

}  // namespace sgf
