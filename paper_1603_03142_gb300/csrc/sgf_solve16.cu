// sgf_solve16.cu -- solve kernels on the register-resident radix-16 FFT
// (sgf_fft16.cuh), N in [16, 4096].
//
// Every P = 2N point transform of the method splits into two N-point "parity
// halves" (even bins: x[n]; odd bins: x[n] W_P^n).  One slot of 16 values per
// thread and per half; a CTA holds both halves of one row pair (row passes),
// or one half of one column (column pass, two CTAs per column in a cluster).
// Operands are staged in shared memory with asynchronous copies (cp.async,
// 16-byte chunks) so that the loads of the next operand overlap the transform
// of the current one; the twiddle table W_N lives in shared memory.
//
//  k_row_fwd16 : sigma rows -> (sigma, dx, dy) with the slope rule and the
//                covered-cell mask, Case-2 phase gather, two rows per complex
//                transform, Hermitian unpack, transposed store.
//  k_col16     : per (column, parity half): forward column transforms of all
//                inputs and fields, spectral multiply-accumulate in registers
//                (the sums of products of Sec. 2.2), inverse transforms; the
//                odd half is folded into the even half through distributed
//                shared memory and the even CTA stores the column.
//  k_row_inv16 : per row pair of a target level: Hermitian extension, inverse
//                row transforms of every contributing output, Case-3 phase
//                interleave, covered cells zeroed, Fx/Fy stored.
#include <cooperative_groups.h>

#include "sgf_fft16.cuh"
#include "sgf_internal.h"

namespace cg = cooperative_groups;

namespace sgf {

template <typename T> struct Cx;
template <> struct Cx<float> { using C = float2; using C2 = float4; };
template <> struct Cx<double> { using C = double2; using C2 = double4_32a; };

// ------------------------------------------------------------ async copies
__device__ __forceinline__ void cp16(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int K>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(K) : "memory"); }

// Whole block: copy `bytes` (a multiple of 16, both ends 16-byte aligned).
__device__ __forceinline__ void cp_block(void *smem, const void *gmem, size_t bytes)
{
    for (size_t o = (size_t)threadIdx.x * 16; o < bytes; o += (size_t)blockDim.x * 16)
        cp16(static_cast<char *>(smem) + o, static_cast<const char *>(gmem) + o);
}

// W_P^n for n = j + u N/16: W_P^j W_32^u from the shared twiddle area.
template <typename C>
__device__ __forceinline__ C twist(const C *tw, const TwLayout &tl, int j, int u)
{
    return hmul(tw[tl.base + j], tw[tl.w32 + u]);
}

// Twiddle area bytes in shared memory (a 16-byte multiple).
template <typename C>
__host__ __device__ __forceinline__ size_t tw_bytes(int entries)
{
    return (((size_t)entries * sizeof(C)) + 15) & ~(size_t)15;
}

template <typename T>
__device__ __forceinline__ bool covered16(const SolveArgs<T> &a, int s, int j, int i)
{
    const int ox = a.child_ox[s];
    if (ox < 0)
        return false;
    const int oy = a.child_oy[s], half = a.N >> 1;
    return i >= ox && i < ox + half && j >= oy && j < oy + half;
}

// ------------------------------------------------------------------ row_fwd
// Shared memory: twiddle area | sigma rows[6][N] | sbuf[2 SP], SP = N + N/16 + 2
// (the pad keeps the two parity halves on different banks in the unpack).
template <typename T>
__global__ void __launch_bounds__(512) k_row_fwd16(SolveArgs<T> a)
{
    using C = typename Cx<T>::C;
    using C2 = typename Cx<T>::C2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = a.N, Q = N >> 4, SP = N + Q + 2;
    C *tw = reinterpret_cast<C *>(smem_raw);
    T *srow = reinterpret_cast<T *>(smem_raw + tw_bytes<C>(a.tw_entries));  // rows ja-1, ja, ja+1, jb-1, jb, jb+1
    C *sbuf = reinterpret_cast<C *>(srow + 6 * N);
    const FwdItem item = a.fwd_items[blockIdx.x];
    const FwdSlab sl = a.slabs[item.slab];
    const int rows = sl.rows, r0 = 2 * item.row_pair;
    const int ja = sl.m * r0 + sl.py, jb = sl.m * (r0 + 1) + sl.py;
    const T *src = a.src[sl.level];
    cp_block(tw, a.tw, tw_bytes<C>(a.tw_entries));
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        const int jr = min(max((q < 3 ? ja : jb) + (q % 3) - 1, 0), N - 1);
        cp_block(srow + q * N, src + (size_t)jr * N, (size_t)N * sizeof(T));
    }
    cp_commit();
    const int t = threadIdx.x;
    const bool active = t < 2 * Q;
    const int b = active ? t / Q : 0, j = active ? t - b * Q : 0;
    Fft16Plan pl;
    pl.init(N, a.logN);
    const TwLayout tl = tw_layout(pl.twlen, N);
    cp_wait<0>();
    __syncthreads();
    C2 *out = reinterpret_cast<C2 *>(a.fwd + sl.off);  // pairs of rows (r0, r0+1)
    for (int f = 0; f < 3; ++f) {
        C v[16];
        if (active) {
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int c = j + u * Q;
                T fv[2] = {T(0), T(0)};
                if (c < rows) {
                    const int i = sl.m * c + sl.px;
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int jj = h ? jb : ja;
                        const T *r = srow + (3 * h + 1) * N;  // row jj; rows jj -+ 1 sit beside it
                        if (covered16(a, sl.level, jj, i))
                            continue;
                        if (f == 0) {
                            fv[h] = r[i];
                        } else if (f == 1) {
                            const int il = i == 0 ? 0 : i - 1, ir = i == N - 1 ? N - 1 : i + 1;
                            const T d = r[ir] - r[il];
                            fv[h] = (ir - il == 2) ? T(0.5) * d : d;
                        } else {
                            const T *rl = jj == 0 ? r : r - N;
                            const T *rr = jj == N - 1 ? r : r + N;
                            const T d = rr[i] - rl[i];
                            fv[h] = (jj == 0 || jj == N - 1) ? d : T(0.5) * d;
                        }
                    }
                }
                C z = hmk<C>(fv[0], fv[1]);
                if (b)
                    z = hmul(z, twist(tw, tl, j, u));
                v[u] = z;
            }
        }
        fft16_block<C, false>(v, sbuf, b, SP, j, active, pl, tw);
        __syncthreads();
        if (active) {
#pragma unroll
            for (int u = 0; u < 16; ++u)
                sbuf[b * SP + pad16(j + u * Q)] = v[u];
        }
        __syncthreads();
        // X_a = (Z + conj Z~)/2, X_b = (Z - conj Z~)/(2i); Z~ = bin -kx, same parity half
        for (int kx = t; kx <= N; kx += blockDim.x) {
            const int bb = kx & 1, k = kx >> 1;
            const int km = (N - bb - k) & (N - 1);
            const C Z = sbuf[bb * SP + pad16(k)];
            const C Zm = sbuf[bb * SP + pad16(km)];
            C2 o;
            o.x = T(0.5) * (Z.x + Zm.x);
            o.y = T(0.5) * (Z.y - Zm.y);
            o.z = T(0.5) * (Z.y + Zm.y);
            o.w = T(-0.5) * (Z.x - Zm.x);
            out[(((size_t)f * (N + 1) + kx) * rows + r0) >> 1] = o;
        }
    }
}

// --------------------------------------------------------------------- col
// Exchange buffer of the column pass, rounded up to a 16-byte multiple.
template <typename C>
__host__ __device__ __forceinline__ size_t col_sbuf_bytes(int N)
{
    return (((size_t)(N + N / 16) * sizeof(C)) + 15) & ~(size_t)15;
}

// Shared memory: twiddle area | sbuf[N + N/16] | stage[2] { column[N] (complex),
// this parity's half of the two spectrum rows, 2 x (N/2 + 4) reals }.
// The odd half's results are folded into the even CTA's stage area at the end.
template <typename T>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(256) k_col16(SolveArgs<T> a)
{
    using C = typename Cx<T>::C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = a.N, Q = N >> 4, QS = quarter_stride(N), HQ = quarter_half(N);
    C *tw = reinterpret_cast<C *>(smem_raw);
    C *sbuf = reinterpret_cast<C *>(smem_raw + tw_bytes<C>(a.tw_entries));
    // the stages take 16-byte asynchronous copies: start them on a 16-byte boundary
    unsigned char *stage_base = reinterpret_cast<unsigned char *>(sbuf) + col_sbuf_bytes<C>(N);
    const size_t stage_bytes = (size_t)N * sizeof(C) + 2 * (size_t)HQ * sizeof(T);
    cg::cluster_group cluster = cg::this_cluster();
    const int b = (int)cluster.block_rank();  // parity half
    const int kx = blockIdx.x >> 1;
    const ColOutput o = a.outs[blockIdx.y];
    const int t = threadIdx.x;
    const bool active = t < Q;
    const int j = active ? t : 0;
    const int nitems = 3 * o.in_count;
    Fft16Plan pl;
    pl.init(N, a.logN);
    const TwLayout tl = tw_layout(pl.twlen, N);
    const int P = 2 * N;

    auto issue = [&](int k) {
        unsigned char *st = stage_base + (size_t)(k & 1) * stage_bytes;
        const ColInput ci = a.ins[o.in_begin + k / 3];
        const FwdSlab sl = a.slabs[ci.slab];
        const int f = k % 3;
        cp_block(st, a.fwd + sl.off + ((size_t)f * (N + 1) + kx) * sl.rows, (size_t)sl.rows * sizeof(C));
        if (ci.kind == SPEC_QUARTER) {
            const T *sp = reinterpret_cast<const T *>(a.spec) + ci.spec_off;
            T *dst = reinterpret_cast<T *>(st + (size_t)N * sizeof(C));
            cp_block(dst, sp + ((size_t)f * (N + 1) + kx) * QS + b * HQ, (size_t)HQ * sizeof(T));
            cp_block(dst + HQ, sp + ((size_t)(3 + f) * (N + 1) + kx) * QS + b * HQ, (size_t)HQ * sizeof(T));
        }
    };
    cp_block(tw, a.tw, tw_bytes<C>(a.tw_entries));
    issue(0);
    cp_commit();
    if (nitems > 1)
        issue(1);
    cp_commit();

    C ax[16], ay[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) {
        ax[u] = hmk<C>(T(0), T(0));
        ay[u] = hmk<C>(T(0), T(0));
    }
    for (int k = 0; k < nitems; ++k) {
        cp_wait<1>();
        __syncthreads();
        const unsigned char *st = stage_base + (size_t)(k & 1) * stage_bytes;
        const C *col = reinterpret_cast<const C *>(st);
        const T *spx = reinterpret_cast<const T *>(st + (size_t)N * sizeof(C));
        const ColInput ci = a.ins[o.in_begin + k / 3];
        const int rows = a.slabs[ci.slab].rows;
        const int f = k % 3;
        C v[16];
        if (active) {
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int n = j + u * Q;
                C x = hmk<C>(T(0), T(0));
                if (n < rows) {
                    x = col[n];
                    if (b)
                        x = hmul(x, twist(tw, tl, j, u));
                }
                v[u] = x;
            }
        }
        fft16_block<C, false>(v, sbuf, 0, N + Q, j, active, pl, tw);
        if (active) {
            if (ci.kind == SPEC_QUARTER) {
                // K0x, K0y imaginary (stored Im), the rest real; bins above N read the
                // quarter at P - ky with the table's ky parity: + K0x Kxx Kyy, - Kxy K0y Kyx.
                // Bin ky = 2k' + b sits at k' of this parity's half row; its mirror
                // P - ky sits at N - k' - b.
                const T mx = (f == 2) ? T(-1) : T(1);
                const T my = (f == 2) ? T(1) : T(-1);
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    const int kp = j + u * Q;
                    const bool hi = 2 * kp + b > N;
                    const int q = hi ? N - kp - b : kp;
                    const T rx = spx[q] * (hi ? mx : T(1));
                    const T ry = spx[HQ + q] * (hi ? my : T(1));
                    C tx = hmk<C>(rx * v[u].x, rx * v[u].y), ty = hmk<C>(ry * v[u].x, ry * v[u].y);
                    if (f == 0) {
                        tx = hmk<C>(-tx.y, tx.x);
                        ty = hmk<C>(-ty.y, ty.x);
                    }
                    ax[u] = hadd(ax[u], tx);
                    ay[u] = hadd(ay[u], ty);
                }
            } else {
                const C *sx = reinterpret_cast<const C *>(a.spec) + ci.spec_off + ((size_t)f * (N + 1) + kx) * P;
                const C *sy = reinterpret_cast<const C *>(a.spec) + ci.spec_off + ((size_t)(3 + f) * (N + 1) + kx) * P;
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    const int ky = 2 * (j + u * Q) + b;
                    ax[u] = hadd(ax[u], hmul(__ldg(sx + ky), v[u]));
                    ay[u] = hadd(ay[u], hmul(__ldg(sy + ky), v[u]));
                }
            }
        }
        __syncthreads();  // stage (k & 1) consumed by every thread
        if (k + 2 < nitems)
            issue(k + 2);
        cp_commit();
    }
    cp_wait<0>();
    // inverse column transforms; y[n] = even[n] + W_P^{-n} odd[n]
    fft16_block<C, true>(ax, sbuf, 0, N + Q, j, active, pl, tw);
    fft16_block<C, true>(ay, sbuf, 0, N + Q, j, active, pl, tw);
    C *fold = reinterpret_cast<C *>(stage_base);  // 2N complex in the even CTA
    cluster.sync();  // the even CTA's stage area is free
    if (b == 1 && active) {
        C *dst = cluster.map_shared_rank(fold, 0);
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const int n = j + u * Q;
            const C w = twist(tw, tl, j, u);
            dst[n] = hmulc(ax[u], w);
            dst[N + n] = hmulc(ay[u], w);
        }
    }
    cluster.sync();
    if (b == 0 && active) {
        C *dst = a.bwd + o.off;
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const int n = j + u * Q;
            if (n < o.rows) {
                dst[bwd_index(N, o.rows, 0, kx, n)] = hadd(ax[u], fold[n]);
                dst[bwd_index(N, o.rows, 1, kx, n)] = hadd(ay[u], fold[N + n]);
            }
        }
    }
}

// ------------------------------------------------------------ zero-rim path
// Forward row pass of a SGF_PLAN_ZERO_RIM plan: the rows of sigma alone (the
// slopes are folded into the merged spectra).  Also verifies the guarantee:
// the CTAs of rows 0-1 and N-2..N-1 scan their rows, every CTA its cells in
// columns 0, 1, N-2, N-1; a nonzero value sets STATUS_RIM_NONZERO.
// Shared memory: twiddle area | sigma rows[2][N] | sbuf[2 SP], SP = N + N/16 + 2.
template <typename T>
__global__ void __launch_bounds__(512) k_row_fwd_m(SolveArgs<T> a)
{
    using C = typename Cx<T>::C;
    using C2 = typename Cx<T>::C2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = a.N, Q = N >> 4, SP = N + Q + 2;
    C *tw = reinterpret_cast<C *>(smem_raw);
    T *srow = reinterpret_cast<T *>(smem_raw + tw_bytes<C>(a.tw_entries));
    C *sbuf = reinterpret_cast<C *>(srow + 2 * N);
    __shared__ int rim_bad;
    const int r0 = 2 * blockIdx.x;
    const T *src = a.src[0] + (size_t)r0 * N;
    cp_block(tw, a.tw, tw_bytes<C>(a.tw_entries));
    cp_block(srow, src, 2 * (size_t)N * sizeof(T));
    cp_commit();
    const int t = threadIdx.x;
    if (t == 0)
        rim_bad = 0;
    const bool active = t < 2 * Q;
    const int b = active ? t / Q : 0, j = active ? t - b * Q : 0;
    Fft16Plan pl;
    pl.init(N, a.logN);
    const TwLayout tl = tw_layout(pl.twlen, N);
    cp_wait<0>();
    __syncthreads();
    {
        bool bad = false;
        if (r0 == 0 || r0 == N - 2) {
            for (int i = t; i < 2 * N; i += blockDim.x)
                bad |= srow[i] != T(0);
        } else if (t < 8) {
            const int col = (t & 3) < 2 ? (t & 3) : N - 4 + (t & 3);  // 0, 1, N-2, N-1
            bad = srow[(t >> 2) * N + col] != T(0);
        }
        if (bad)
            rim_bad = 1;
    }
    C v[16];
    if (active) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const int c = j + u * Q;
            C z = hmk<C>(srow[c], srow[N + c]);
            if (b)
                z = hmul(z, twist(tw, tl, j, u));
            v[u] = z;
        }
    }
    fft16_block<C, false>(v, sbuf, b, SP, j, active, pl, tw);
    __syncthreads();
    if (t == 0 && rim_bad)
        atomicOr(a.status, STATUS_RIM_NONZERO);
    if (active) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
            sbuf[b * SP + pad16(j + u * Q)] = v[u];
    }
    __syncthreads();
    C2 *out = reinterpret_cast<C2 *>(a.fwd);
    for (int kx = t; kx <= N; kx += blockDim.x) {
        const int bb = kx & 1, k = kx >> 1;
        const int km = (N - bb - k) & (N - 1);
        const C Z = sbuf[bb * SP + pad16(k)];
        const C Zm = sbuf[bb * SP + pad16(km)];
        C2 o;
        o.x = T(0.5) * (Z.x + Zm.x);
        o.y = T(0.5) * (Z.y - Zm.y);
        o.z = T(0.5) * (Z.y + Zm.y);
        o.w = T(-0.5) * (Z.x - Zm.x);
        out[((size_t)kx * N + r0) >> 1] = o;
    }
}

// Column pass of a SGF_PLAN_ZERO_RIM plan: one forward transform, the two
// merged spectra (Fx^ = Gx^ sigma^, Fy^ = Gy^ sigma^, both imaginary), two
// inverse transforms; parity halves folded through distributed shared memory.
// Two CTAs per SM.  Shared memory: twiddle area | sbuf[N + N/16] | stage
// {column[N], this parity's half rows of Gx and Gy}; the fold reuses sbuf+stage.
template <typename T>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(256, sizeof(T) == 4 ? 2 : 1) k_col_m(SolveArgs<T> a)
{
    using C = typename Cx<T>::C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = a.N, Q = N >> 4, QS = quarter_stride(N), HQ = quarter_half(N);
    C *tw = reinterpret_cast<C *>(smem_raw);
    C *sbuf = reinterpret_cast<C *>(smem_raw + tw_bytes<C>(a.tw_entries));
    unsigned char *stage = reinterpret_cast<unsigned char *>(sbuf) + col_sbuf_bytes<C>(N);
    C *col = reinterpret_cast<C *>(stage);
    T *gsp = reinterpret_cast<T *>(stage + (size_t)N * sizeof(C));
    cg::cluster_group cluster = cg::this_cluster();
    const int b = (int)cluster.block_rank();
    const int kx = blockIdx.x >> 1;
    const int t = threadIdx.x;
    const bool active = t < Q;
    const int j = active ? t : 0;
    Fft16Plan pl;
    pl.init(N, a.logN);
    const TwLayout tl = tw_layout(pl.twlen, N);
    const T *spec = reinterpret_cast<const T *>(a.spec);
    cp_block(tw, a.tw, tw_bytes<C>(a.tw_entries));
    cp_block(col, a.fwd + (size_t)kx * N, (size_t)N * sizeof(C));
    cp_block(gsp, spec + (size_t)kx * QS + b * HQ, (size_t)HQ * sizeof(T));
    cp_block(gsp + HQ, spec + ((size_t)(N + 1) + kx) * QS + b * HQ, (size_t)HQ * sizeof(T));
    cp_commit();
    cp_wait<0>();
    __syncthreads();
    C ax[16], ay[16];
    {
        C v[16];
        if (active) {
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                C x = col[j + u * Q];
                if (b)
                    x = hmul(x, twist(tw, tl, j, u));
                v[u] = x;
            }
        }
        fft16_block<C, false>(v, sbuf, 0, N + Q, j, active, pl, tw);
        if (active) {
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int kp = j + u * Q;
                const bool hi = 2 * kp + b > N;
                const int q = hi ? N - kp - b : kp;
                const T gx = gsp[q];                           // Gx even in ky
                const T gy = hi ? -gsp[HQ + q] : gsp[HQ + q];  // Gy odd in ky
                ax[u] = hmk<C>(-gx * v[u].y, gx * v[u].x);     // i gx v
                ay[u] = hmk<C>(-gy * v[u].y, gy * v[u].x);
            }
        }
    }
    fft16_block<C, true>(ax, sbuf, 0, N + Q, j, active, pl, tw);
    fft16_block<C, true>(ay, sbuf, 0, N + Q, j, active, pl, tw);
    C *fold = sbuf;  // 2N complex over sbuf and the stage (both free after the transforms)
    cluster.sync();
    if (b == 1 && active) {
        C *dst = cluster.map_shared_rank(fold, 0);
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const int n = j + u * Q;
            const C w = twist(tw, tl, j, u);
            dst[n] = hmulc(ax[u], w);
            dst[N + n] = hmulc(ay[u], w);
        }
    }
    cluster.sync();
    if (b == 0 && active) {
        C *dst = a.bwd;
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const int n = j + u * Q;
            dst[bwd_index(N, N, 0, kx, n)] = hadd(ax[u], fold[n]);
            dst[bwd_index(N, N, 1, kx, n)] = hadd(ay[u], fold[N + n]);
        }
    }
}

// ------------------------------------------------------------------ row_inv
// The two rows of every (contribution, component) are gathered as 32-byte
// pieces (4 bins of one row, tiled output layout) with asynchronous copies
// into a staging buffer; the next gather is issued as soon as the current one
// has been read into registers, so it overlaps the inverse transform.
// Shared memory: twiddle area | stage[2 rows][N/4 + 1][4] | sbuf[2 SP] | O[2 comps][2 rows][N].
template <typename T>
__global__ void __launch_bounds__(512) k_row_inv16(SolveArgs<T> a)
{
    using C = typename Cx<T>::C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = a.N, Q = N >> 4, SP = N + Q + 2, P = 2 * N, G = N / 4 + 1;
    C *tw = reinterpret_cast<C *>(smem_raw);
    C *stg = reinterpret_cast<C *>(smem_raw + tw_bytes<C>(a.tw_entries));  // [row][G][4]
    C *sbuf = stg + 2 * 4 * G;
    T *O = reinterpret_cast<T *>(sbuf + 2 * SP);
    const int tl = blockIdx.y;
    const int j0 = 2 * blockIdx.x, j1 = j0 + 1;
    const int t = threadIdx.x;
    const bool active = t < 2 * Q;
    const int b = active ? t / Q : 0, j = active ? t - b * Q : 0;
    Fft16Plan pl;
    pl.init(N, a.logN);
    const TwLayout twl = tw_layout(pl.twlen, N);
    const int c0 = a.contrib_begin[tl], c1 = a.contrib_begin[tl + 1];
    const int nitems = 2 * (c1 - c0);  // (contribution, component)

    // gather item k: rows j0 and j1 of component k % 2 of contribution c0 + k / 2
    auto issue = [&](int k) {
        const RowContrib rc = a.contribs[c0 + k / 2];
        const int comp = k & 1;
        const ColOutput oa = a.outs[rc.out_base + (j0 % rc.m) * rc.m];
        const ColOutput ob = a.outs[rc.out_base + (j1 % rc.m) * rc.m];
        const int ra = j0 / rc.m, rb = j1 / rc.m;
        constexpr int PG = 4 * (int)sizeof(C) / 16;  // 16-byte pieces per group of 4 bins
        constexpr int EP = 16 / (int)sizeof(C);      // bins per piece
        for (int q = t; q < 2 * G * PG; q += blockDim.x) {
            const int row = q / (G * PG), rem = q - row * G * PG, g = rem / PG, piece = rem - g * PG;
            const ColOutput &o = row ? ob : oa;
            const C *src = a.bwd + o.off + bwd_index(N, o.rows, comp, 4 * g, row ? rb : ra) + piece * EP;
            cp16(stg + ((size_t)row * G + g) * 4 + piece * EP, src);
        }
    };
    cp_block(tw, a.tw, tw_bytes<C>(a.tw_entries));
    if (nitems > 0)
        issue(0);
    cp_commit();
    for (int i = t; i < 4 * N; i += blockDim.x)
        O[i] = T(0);
    for (int k = 0; k < nitems; ++k) {
        const RowContrib rc = a.contribs[c0 + k / 2];
        const int comp = k & 1;
        const int nout = N / rc.m;
        cp_wait<0>();
        __syncthreads();
        C v[16];
        if (active) {
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int kx = 2 * (j + u * Q) + b;
                const int k2 = kx <= N ? kx : P - kx;
                const C A = stg[k2], B = stg[4 * G + k2];
                // Z = A + iB, from the stored half (kx <= N) or its conjugate mirror
                v[u] = kx <= N ? hmk<C>(A.x - B.y, A.y + B.x) : hmk<C>(A.x + B.y, B.x - A.y);
            }
        }
        __syncthreads();  // the stage has been read
        if (k + 1 < nitems)
            issue(k + 1);
        cp_commit();
        fft16_block<C, true>(v, sbuf, b, SP, j, active, pl, tw);
        __syncthreads();
        if (active && b == 1) {
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int n = j + u * Q;
                sbuf[pad16(n)] = hmulc(v[u], twist(tw, twl, j, u));
            }
        }
        __syncthreads();
        if (active && b == 0) {
            T *Oc = O + comp * 2 * N;
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int n = j + u * Q;
                if (n < nout) {
                    const C y = hadd(v[u], sbuf[pad16(n)]);
                    const int i = rc.m * n + rc.px;
                    Oc[i] += y.x;
                    Oc[N + i] += y.y;
                }
            }
        }
    }
    __syncthreads();
    T *fx = a.fx[tl], *fy = a.fy[tl];
    for (int i = t; i < N; i += blockDim.x) {
        const bool ca = covered16(a, tl, j0, i), cb = covered16(a, tl, j1, i);
        fx[(size_t)j0 * N + i] = ca ? T(0) : O[i];
        fx[(size_t)j1 * N + i] = cb ? T(0) : O[N + i];
        fy[(size_t)j0 * N + i] = ca ? T(0) : O[2 * N + i];
        fy[(size_t)j1 * N + i] = cb ? T(0) : O[3 * N + i];
    }
}

// ---------------------------------------------------------------- launchers
static inline int warps_up(int n) { return ((n < 32 ? 32 : n) + 31) / 32 * 32; }

template <typename T>
static int tw_entries_for(int N)
{
    int logN = 0;
    while ((1 << logN) < N)
        ++logN;
    Fft16Plan pl;
    pl.init(N, logN);
    return tw_layout(pl.twlen, N).entries;
}
template <typename T>
static size_t smem_fwd16(int N)
{
    using C = typename Cx<T>::C;
    return tw_bytes<C>(tw_entries_for<T>(N)) + 6 * (size_t)N * sizeof(T) + 2 * (size_t)(N + N / 16 + 2) * sizeof(C);
}
template <typename T>
static size_t smem_col16(int N)
{
    using C = typename Cx<T>::C;
    const size_t stage = (size_t)N * sizeof(C) + 2 * (size_t)quarter_half(N) * sizeof(T);
    return tw_bytes<C>(tw_entries_for<T>(N)) + col_sbuf_bytes<C>(N) + 2 * stage;  // 2 stages >= 2N complex (fold)
}
template <typename T>
static size_t smem_inv16(int N)
{
    using C = typename Cx<T>::C;
    return tw_bytes<C>(tw_entries_for<T>(N)) + 2 * 4 * (size_t)(N / 4 + 1) * sizeof(C) +
           2 * (size_t)(N + N / 16 + 2) * sizeof(C) + 4 * (size_t)N * sizeof(T);
}

template <typename T>
cudaError_t merged_init();

template <typename T>
cudaError_t solve16_init()
{
    const int maxN = sizeof(T) == 8 ? 2048 : 4096;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_row_fwd16<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem_fwd16<T>(maxN))) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k_col16<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem_col16<T>(maxN))) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k_row_inv16<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem_inv16<T>(maxN))) != cudaSuccess)
        return e;
    return merged_init<T>();
}

template <typename T>
cudaError_t launch_row_fwd16(const SolveArgs<T> &a, int n_items, cudaStream_t st)
{
    k_row_fwd16<T><<<n_items, warps_up(2 * (a.N / 16)), smem_fwd16<T>(a.N), st>>>(a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_col16(const SolveArgs<T> &a, int n_outputs, cudaStream_t st)
{
    dim3 grid(2 * (a.N + 1), n_outputs);
    k_col16<T><<<grid, warps_up(a.N / 16), smem_col16<T>(a.N), st>>>(a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_row_inv16(const SolveArgs<T> &a, cudaStream_t st)
{
    dim3 grid(a.N / 2, a.L);
    k_row_inv16<T><<<grid, warps_up(2 * (a.N / 16)), smem_inv16<T>(a.N), st>>>(a);
    return cudaGetLastError();
}

template <typename T>
static size_t smem_fwd_m(int N)
{
    using C = typename Cx<T>::C;
    return tw_bytes<C>(tw_entries_for<T>(N)) + 2 * (size_t)N * sizeof(T) + 2 * (size_t)(N + N / 16 + 2) * sizeof(C);
}
template <typename T>
static size_t smem_col_m(int N)
{
    using C = typename Cx<T>::C;
    size_t stage = (size_t)N * sizeof(C) + 2 * (size_t)quarter_half(N) * sizeof(T);
    const size_t sb = col_sbuf_bytes<C>(N);
    if (sb + stage < 2 * (size_t)N * sizeof(C))  // the fold spans sbuf and the stage
        stage = 2 * (size_t)N * sizeof(C) - sb;
    return tw_bytes<C>(tw_entries_for<T>(N)) + sb + stage;
}

template <typename T>
cudaError_t merged_init()
{
    const int maxN = sizeof(T) == 8 ? 2048 : 4096;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_row_fwd_m<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem_fwd_m<T>(maxN))) != cudaSuccess)
        return e;
    return cudaFuncSetAttribute(k_col_m<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_col_m<T>(maxN));
}

template <typename T>
cudaError_t launch_row_fwd_merged(const SolveArgs<T> &a, cudaStream_t st)
{
    k_row_fwd_m<T><<<a.N / 2, warps_up(2 * (a.N / 16)), smem_fwd_m<T>(a.N), st>>>(a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_col_merged(const SolveArgs<T> &a, cudaStream_t st)
{
    k_col_m<T><<<2 * (a.N + 1), warps_up(a.N / 16), smem_col_m<T>(a.N), st>>>(a);
    return cudaGetLastError();
}

template cudaError_t launch_row_fwd_merged<float>(const SolveArgs<float> &, cudaStream_t);
template cudaError_t launch_row_fwd_merged<double>(const SolveArgs<double> &, cudaStream_t);
template cudaError_t launch_col_merged<float>(const SolveArgs<float> &, cudaStream_t);
template cudaError_t launch_col_merged<double>(const SolveArgs<double> &, cudaStream_t);

template cudaError_t solve16_init<float>();
template cudaError_t solve16_init<double>();
template cudaError_t launch_row_fwd16<float>(const SolveArgs<float> &, int, cudaStream_t);
template cudaError_t launch_row_fwd16<double>(const SolveArgs<double> &, int, cudaStream_t);
template cudaError_t launch_col16<float>(const SolveArgs<float> &, int, cudaStream_t);
template cudaError_t launch_col16<double>(const SolveArgs<double> &, int, cudaStream_t);
template cudaError_t launch_row_inv16<float>(const SolveArgs<float> &, cudaStream_t);
template cudaError_t launch_row_inv16<double>(const SolveArgs<double> &, cudaStream_t);

}  // namespace sgf
