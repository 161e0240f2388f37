// sgf_kernels.cuh -- solve kernels on the register-resident radix-16 FFT,
// templated on log2(N) so that every stride and index folds at compile time.
// Instantiated once per N by sgf_inst_<logN>.cu; dispatched by sgf_dispatch.cu.
//
// Every P = 2N point transform of the method splits into two N-point "parity
// halves" (even bins: x[n]; odd bins: x[n] W_P^n).  One slot of 16 values per
// thread and per half; a CTA holds both halves of one row pair (row passes),
// or one half of one column (column passes: two CTAs per column in a cluster,
// the odd half folded into the even one through distributed shared memory).
// Operands are staged in shared memory with asynchronous copies (cp.async,
// 16-byte chunks) so that loads overlap transforms; twiddles live in shared
// memory (sgf_fft16.cuh, TwLayout).
//
//  k_row_fwd   : sigma rows -> (sigma, dx, dy) with the slope rule and the
//                covered-cell mask, Case-2 phase gather, two rows per complex
//                transform, Hermitian unpack, transposed store.
//  k_col       : per (column, parity half): forward column transforms of all
//                inputs and fields, spectral multiply-accumulate in registers
//                (the sums of products of Sec. 2.2), inverse transforms.
//  k_col_g     : the Case-3 phase outputs of one (coarser source, target)
//                pair together: source fields transformed once per column.
//  k_col_sum   : outputs with long input lists, split into chunks of k_col work
//                items: chunk accumulators summed in order, transformed back.
//  k_row_inv   : per row pair of a target level: Hermitian extension, inverse
//                row transforms of every contributing output, Case-3 phase
//                interleave, covered cells zeroed, Fx/Fy stored.
//  k_row_inv1  : k_row_inv for a level whose only contribution is its own
//                main output (level 0), one CTA per (row pair, component).
//  k_row_fwd_m,
//  k_col_m     : the SGF_PLAN_ZERO_RIM variants (sigma alone, merged spectra);
//  k_col_md    : k_col_m with both inverse transforms in flight (another
//                schedule of the same arithmetic, chosen by the autotuner).
#pragma once
#include <atomic>
#include <type_traits>
#include <cooperative_groups.h>

#include "sgf_fft16.cuh"
#include "sgf_internal.h"

namespace sgf {

namespace cg = cooperative_groups;

template <typename T> struct Cx;
template <> struct Cx<float> { using C = float2; using C2 = float4; };
template <> struct Cx<double> { using C = double2; using C2 = double4_32a; };

// ------------------------------------------------------------ async copies
__device__ __forceinline__ void cp16(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp8(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
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

// Twiddle area bytes in shared memory (a 16-byte multiple).
template <typename C>
__host__ __device__ __forceinline__ size_t tw_bytes(int entries)
{
    return (((size_t)entries * sizeof(C)) + 15) & ~(size_t)15;
}

// cos and sin of 2 pi u / 32, u = 0..15.
__device__ constexpr double kW32c[16] = {
    1.0, 0.98078528040323044913, 0.92387953251128675613, 0.83146961230254523708,
    0.70710678118654752440, 0.55557023301960222474, 0.38268343236508977173, 0.19509032201612826785,
    0.0, -0.19509032201612826785, -0.38268343236508977173, -0.55557023301960222474,
    -0.70710678118654752440, -0.83146961230254523708, -0.92387953251128675613, -0.98078528040323044913};
__device__ constexpr double kW32s[16] = {
    0.0, 0.19509032201612826785, 0.38268343236508977173, 0.55557023301960222474,
    0.70710678118654752440, 0.83146961230254523708, 0.92387953251128675613, 0.98078528040323044913,
    1.0, 0.98078528040323044913, 0.92387953251128675613, 0.83146961230254523708,
    0.70710678118654752440, 0.55557023301960222474, 0.38268343236508977173, 0.19509032201612826785};

// W_P^n for n = j + u N/16 (P = 2N): W_P^j from the shared twiddle area times
// W_32^u = cos(2 pi u/32) - i sin(2 pi u/32), a constant (u is unrolled at
// every call).
template <typename C>
__device__ __forceinline__ C twist(const C *tw, const TwLayout &tl, int j, int u)
{
    using T = typename Real<C>::T;
    return hmul(tw[tl.base + j], hmk<C>((T)kW32c[u], (T)-kW32s[u]));
}

// Sequence stride (complex) of a column-pass exchange buffer: N + N/16 rounded
// up so the next buffer starts on a 16-byte boundary.
template <typename C>
__host__ __device__ constexpr int col_sp(int N)
{
    return (int)(((((size_t)(N + N / 16) * sizeof(C)) + 15) & ~(size_t)15) / sizeof(C));
}

// Is cell (i, j) of patch s under a patch of the next finer level?
template <typename T>
__device__ __forceinline__ bool covered(const SolveArgs<T> &a, int s, int j, int i)
{
    for (int k = a.cover_begin[s]; k < a.cover_begin[s + 1]; ++k) {
        const CoverRect &r = a.cover[k];
        if (i >= r.x0 && i < r.x1 && j >= r.y0 && j < r.y1)
            return true;
    }
    return false;
}

template <int LOGN>
struct KShape {
    static constexpr int N = 1 << LOGN, Q = N >> 4;
    static constexpr int ROW_THREADS = 2 * Q < 32 ? 32 : 2 * Q;  // both parity halves
    static constexpr int COL_THREADS = Q < 32 ? 32 : Q;          // one parity half
    static constexpr int SP_ROW = N + Q + 8;  // pad puts the two halves 16 banks apart for the unpack
    // threads per parity half for the half barriers of the row kernels (0: whole-block barriers)
    static constexpr int HB_ROW = Q >= 32 ? Q : 0;
};

// Tensor-core tiles (SGF_BF16X) issued per round, i.e. A-tile buffers in shared
// memory: all of them, except where the kernel's own staging leaves no room at
// N = 4096 (k_row_fwd keeps two; k_row_inv keeps one and is never launched
// there: the host refuses SGF_BF16X nests of N = 4096 with more than one level).
enum : int {
    KK_ROW_FWD,
    KK_COL,
    KK_ROW_INV,
    KK_ROW_INV1,
    KK_ROW_FWD_M,
    KK_COL_M,
    KK_COL_MD,
    KK_COL_G,
    KK_COL_SUM,
    KK_ROW_INV2,
    KK_COL_MW
};
__host__ __device__ constexpr int tc_round(int logn, int tiles, int kind)
{
    return logn < 12                                 ? tiles
           : kind == KK_ROW_FWD                      ? (tiles < 2 ? tiles : 2)
           : kind == KK_ROW_INV || kind == KK_COL_G || kind == KK_ROW_INV2 || kind == KK_COL_MW ? 1
                                                                          : tiles;
}

// ------------------------------------------------------------------ row_fwd
// One CTA per (row pair, field): field f = blockIdx.y of (sigma, x slope, y
// slope).  The rows it needs (ja and jb; for the y slope the rows either side of
// each, clamped at the patch edge where the slope is one-sided) are staged in
// the exchange buffers' space and read before the transform, so a CTA holds the
// twiddles and the exchange buffers only (two CTAs per SM in FP32).
// Shared memory: twiddle area | sbuf[2 SP_ROW] (first the staged rows).
template <typename T, int LOGN, bool BATCH, bool TC>
__global__ void __launch_bounds__(KShape<LOGN>::ROW_THREADS, sizeof(T) == 4 && !TC ? 2 : 1)
    k_row_fwd(SolveArgs<T> a0, BatchView<T> bv)
{
    const int2 wm = BATCH ? bv.map[blockIdx.x] : make_int2(0, (int)blockIdx.x);
    const SolveArgs<T> &a = BATCH ? bv.args[wm.x] : a0;
    using C = typename Cx<T>::C;
    using C2 = typename Cx<T>::C2;
    using K = KShape<LOGN>;
    constexpr int N = K::N, Q = K::Q, SP = K::SP_ROW;
    extern __shared__ __align__(16) unsigned char smem_tc[];
    constexpr int TCT = tc_tiles(KShape<LOGN>::ROW_THREADS, 1);
    constexpr int TCR = tc_round(LOGN, TCT, KK_ROW_FWD);
    static_assert(!TC || sizeof(T) == 4, "tensor-core tiles take FP32 data");
    unsigned char *smem_raw = smem_tc + (TC ? tc_smem_bytes(TCR) : 0);
    TcCtx tcx;
    if constexpr (TC)
        tc_begin(tcx, smem_tc, TCT, TCR, a.status, a.wait_cycles, a.inject);
    C *tw = reinterpret_cast<C *>(smem_raw);
    C *sbuf = reinterpret_cast<C *>(smem_raw + tw_bytes<C>(a.tw_entries));
    T *srow = reinterpret_cast<T *>(sbuf);  // f < 2: rows ja, jb; f = 2: ja-1, ja+1, jb-1, jb+1
    const int f = (int)blockIdx.y;
    const FwdItem item = a.fwd_items[wm.y];
    const FwdSlab sl = a.slabs[item.slab];
    const int rows = sl.rows, r0 = 2 * item.row_pair;
    const int ja = sl.m * r0 + sl.py, jb = sl.m * (r0 + 1) + sl.py;
    const T *src = a.src[sl.patch];
    cp_block(tw, a.tw, tw_bytes<C>(a.tw_entries));
    const int nl = a.n_log;  // the patch's own cells a side (<= N; zero beyond, slopes one-sided on its edges)
    if (f < 2) {
        cp_block(srow, src + (size_t)ja * N, (size_t)N * sizeof(T));
        cp_block(srow + N, src + (size_t)jb * N, (size_t)N * sizeof(T));
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int jj = q < 2 ? ja : jb;
            const int jr = (q & 1) ? min(jj + 1, nl - 1) : max(jj - 1, 0);
            cp_block(srow + q * N, src + (size_t)min(jr, N - 1) * N, (size_t)N * sizeof(T));
        }
    }
    cp_commit();
    const int t = threadIdx.x;
    const bool active = t < 2 * Q;
    const int b = active ? t / Q : 0, j = active ? t - b * Q : 0;
    const TwLayout tl = tw_layout(F16<LOGN>::twlen, N);
    cp_wait<0>();
    __syncthreads();
    C v[1][16];
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
                    if (i >= nl || jj >= nl || covered(a, sl.patch, jj, i))
                        continue;
                    if (f == 0) {
                        fv[h] = srow[h * N + i];
                    } else if (f == 1) {
                        const T *r = srow + h * N;
                        const int il = i == 0 ? 0 : i - 1, ir = i == nl - 1 ? nl - 1 : i + 1;
                        const T d = r[ir] - r[il];
                        fv[h] = (ir - il == 2) ? T(0.5) * d : d;
                    } else {
                        const T d = srow[(2 * h + 1) * N + i] - srow[2 * h * N + i];
                        fv[h] = (jj == 0 || jj == nl - 1) ? d : T(0.5) * d;
                    }
                }
            }
            C z = hmk<C>(fv[0], fv[1]);
            if (b)
                z = hmul(z, twist(tw, tl, j, u));
            v[0][u] = z;
        }
    }
    __syncthreads();  // the staged rows are read: the exchange buffers overwrite them
    constexpr int HB = TC ? 0 : K::HB_ROW;
    fft_ct<C, false, LOGN, 1, TC, HB>(v, sbuf + b * SP, SP, j, active, tw, &tcx, b);
    __syncthreads();
    if (active) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
            sbuf[b * SP + pad16(j + u * Q)] = v[0][u];
    }
    __syncthreads();
    // X_a = (Z + conj Z~)/2, X_b = (Z - conj Z~)/(2i); Z~ = bin -kx, same parity half
    C2 *out = reinterpret_cast<C2 *>(a.fwd + sl.off);  // pairs of rows (r0, r0+1)
    for (int kx = t; kx <= N; kx += K::ROW_THREADS) {
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
    if constexpr (TC)
        tc_end(tcx, TCT);
}

// ----------------------------------------------------------------- row_fwd2
// k_row_fwd (FP32, no tensor-core tiles, no batch view) with two work items
// (row pairs) per CTA and the three fields (sigma, x slope, y slope) of both in
// the one CTA, one field after the other: the source rows are read once per
// CTA from global memory (the slopes' neighbours from the L1 cache) instead of
// once per field CTA, and in the store phase two neighbouring lanes write the
// two items' values of one bin, 32 contiguous bytes where the items are
// neighbouring row pairs of one slab (every item of a slab with an even number
// of row pairs).  Group g = t / (N/8) of 2 N/16 threads takes item
// 2 blockIdx.x + g (parity halves on named barriers 1 + 2 g + half); a group
// without an item (an odd item count) only keeps the block barriers.  The
// field values are those of k_row_fwd, expression for expression.
// Shared memory: twiddle area | sbuf [2 items][2 halves][SP_ROW].
template <int LOGN>
__global__ void __launch_bounds__((1 << LOGN) / 4) k_row_fwd2(const __grid_constant__ SolveArgs<float> a, int items)
{
    using C = float2;
    using C2 = float4;
    using K = KShape<LOGN>;
    constexpr int N = K::N, Q = K::Q, SP = K::SP_ROW, T2 = 2 * Q;
    static_assert(Q >= 32, "whole warps per parity half");
    extern __shared__ __align__(16) unsigned char smem_f3[];
    C *tw = reinterpret_cast<C *>(smem_f3);
    C *sbuf = reinterpret_cast<C *>(smem_f3 + tw_bytes<C>(a.tw_entries));
    cp_block(tw, a.tw, tw_bytes<C>(a.tw_entries));
    cp_commit();
    const int t = threadIdx.x;
    const int g = t / T2, tg = t - g * T2, b = tg / Q, j = tg - b * Q;
    const int item_g = 2 * (int)blockIdx.x + g;
    const bool active = item_g < items;
    const FwdItem item = a.fwd_items[active ? item_g : 0];
    const FwdSlab sl = a.slabs[item.slab];
    const int rows = sl.rows, r0 = 2 * item.row_pair;
    const int ja = sl.m * r0 + sl.py, jb = sl.m * (r0 + 1) + sl.py;
    const float *src = a.src[sl.patch];
    const int nl = a.n_log;
    // the other group's slab (its store addresses)
    const int item_o = 2 * (int)blockIdx.x + (g ^ 1);
    const TwLayout tl = tw_layout(F16<LOGN>::twlen, N);
    cp_wait<0>();
    __syncthreads();
    auto field = [&](auto fcv) {  // one field after the other, each compiled on its own
        constexpr int f = decltype(fcv)::value;
        C v[1][16];
        if (active) {  // the field's 16 inputs of this thread's slot
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int c = j + u * Q;
                float fv[2] = {0.0f, 0.0f};
                if (c < rows) {
                    const int i = sl.m * c + sl.px;
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int jj = h ? jb : ja;
                        if (i >= nl || jj >= nl || covered(a, sl.patch, jj, i))
                            continue;
                        const float *r = src + (size_t)jj * N;
                        if constexpr (f == 0) {
                            fv[h] = __ldg(r + i);
                        } else if constexpr (f == 1) {
                            const int il = i == 0 ? 0 : i - 1, ir = i == nl - 1 ? nl - 1 : i + 1;
                            const float d = __ldg(r + ir) - __ldg(r + il);
                            fv[h] = (ir - il == 2) ? 0.5f * d : d;
                        } else {
                            const int jd = max(jj - 1, 0), ju = min(jj + 1, nl - 1);
                            const float d = __ldg(src + (size_t)min(ju, N - 1) * N + i) -
                                            __ldg(src + (size_t)min(jd, N - 1) * N + i);
                            fv[h] = (jj == 0 || jj == nl - 1) ? d : 0.5f * d;
                        }
                    }
                }
                C z = hmk<C>(fv[0], fv[1]);
                if (b)
                    z = hmul(z, twist(tw, tl, j, u));
                v[0][u] = z;
            }
        }
        fft_ct<C, false, LOGN, 1, false, Q>(v, sbuf + (2 * g + b) * SP, SP, j, active, tw, nullptr, 2 * g + b);
        __syncthreads();
        if (active) {
#pragma unroll
            for (int u = 0; u < 16; ++u)
                sbuf[(2 * g + b) * SP + pad16(j + u * Q)] = v[0][u];
        }
        __syncthreads();
        // X_a = (Z + conj Z~)/2, X_b = (Z - conj Z~)/(2i); Z~ = bin -kx, same parity half
        for (int e = t; e < 2 * (N + 1); e += 4 * Q) {  // e = 2 kx + item: neighbouring lanes, one sector
            const int pr = e & 1, kx = e >> 1;
            const int it = 2 * (int)blockIdx.x + pr;
            if (it >= items)
                continue;
            const FwdItem ip = pr == g ? item : a.fwd_items[item_o];
            const FwdSlab sp = pr == g ? sl : a.slabs[ip.slab];
            const int bb = kx & 1, k = kx >> 1;
            const int km = (N - bb - k) & (N - 1);
            const C Z = sbuf[(2 * pr + bb) * SP + pad16(k)];
            const C Zm = sbuf[(2 * pr + bb) * SP + pad16(km)];
            C2 o;
            o.x = 0.5f * (Z.x + Zm.x);
            o.y = 0.5f * (Z.y - Zm.y);
            o.z = 0.5f * (Z.y + Zm.y);
            o.w = -0.5f * (Z.x - Zm.x);
            C2 *out = reinterpret_cast<C2 *>(a.fwd + sp.off);  // pairs of rows (r0, r0+1)
            out[(((size_t)f * (N + 1) + kx) * sp.rows + 2 * ip.row_pair) >> 1] = o;
        }
        __syncthreads();  // sbuf is free for the next field's exchanges
    };
    field(std::integral_constant<int, 0>{});
    field(std::integral_constant<int, 1>{});
    field(std::integral_constant<int, 2>{});
}

// --------------------------------------------------------------------- col
// Bytes of one k_col input stage: the column, then this parity's half of the
// quarter spectrum rows or, for FP32 data with N <= 1024, this parity's bins of
// the full complex spectrum rows of an input of Cases 2 and 3 (x and y tables,
// N bins each, gathered from every other bin), copied in ahead like the column
// instead of being loaded in the product.  Not in the tensor-core instances:
// there the larger stage costs more in resident clusters than it saves.
template <typename T, int LOGN, bool TC>
struct ColStage {
    using C = typename Cx<T>::C;
    static constexpr int N = 1 << LOGN;
    static constexpr bool FULL = sizeof(T) == 4 && LOGN <= 10 && !TC;
    static constexpr size_t QB = 2 * (size_t)quarter_half(N) * sizeof(T);
    static constexpr size_t FB = FULL ? 2 * (size_t)N * sizeof(C) : 0;
    static constexpr size_t BYTES = (size_t)N * sizeof(C) + (QB > FB ? QB : FB);
};

// One 2-CTA cluster (the parity halves) per (column, work item); the
// tensor-core instance takes kColWalk columns per cluster.
// Shared memory: twiddle area | sbuf[SPC] | stage[2] { column[N] (complex),
// this parity's half of the two spectrum rows, 2 x (N/2 + 4) reals, or (see
// ColStage) this parity's bins of the full rows [x, y][N] complex }.  The
// dual inverse transform uses sbuf and the stages as two sequence buffers, and
// the fold of the odd half reuses them afterwards.
constexpr int kColWalk = 4;
template <typename T, int LOGN, bool BATCH, bool TC>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(KShape<LOGN>::COL_THREADS) k_col(SolveArgs<T> a0, BatchView<T> bv)
{
    const int2 wm = BATCH ? bv.map[blockIdx.y] : make_int2(0, (int)blockIdx.y);
    const SolveArgs<T> &a = BATCH ? bv.args[wm.x] : a0;
    using C = typename Cx<T>::C;
    using K = KShape<LOGN>;
    constexpr int N = K::N, Q = K::Q, P = 2 * N, QS = quarter_stride(N), HQ = quarter_half(N);
    constexpr int SPC = col_sp<C>(N);
    extern __shared__ __align__(16) unsigned char smem_tc[];
    constexpr int TCT = tc_tiles(KShape<LOGN>::COL_THREADS, 2);
    constexpr int TCR = tc_round(LOGN, TCT, KK_COL);
    static_assert(!TC || sizeof(T) == 4, "tensor-core tiles take FP32 data");
    unsigned char *smem_raw = smem_tc + (TC ? tc_smem_bytes(TCR) : 0);
    TcCtx tcx;
    if constexpr (TC)
        tc_begin(tcx, smem_tc, TCT, TCR, a.status, a.wait_cycles, a.inject);
    C *tw = reinterpret_cast<C *>(smem_raw);
    C *sbuf = reinterpret_cast<C *>(smem_raw + tw_bytes<C>(a.tw_entries));
    unsigned char *stage_base = reinterpret_cast<unsigned char *>(sbuf + SPC);
    using CS = ColStage<T, LOGN, TC>;
    constexpr size_t stage_bytes = CS::BYTES;
    cg::cluster_group cluster = cg::this_cluster();
    const int b = (int)cluster.block_rank();  // parity half
    const ColWork w = a.col_list[wm.y];
    const ColOutput o = a.outs[w.out];
    const int t = threadIdx.x;
    const bool active = t < Q;
    const int j = active ? t : 0;
    const int nitems = 3 * w.in_count;
    const TwLayout tl = tw_layout(F16<LOGN>::twlen, N);
    cp_block(tw, a.tw, tw_bytes<C>(a.tw_entries));
    // tensor-core instances: a cluster takes kColWalk columns of its work item, gridDim.x / 2
    // apart (the tiles, the tensor memory and the twiddles set up once for them)
    constexpr bool WALK = TC && !BATCH;
    for (int kx = blockIdx.x >> 1; kx <= N; kx += WALK ? (int)(gridDim.x >> 1) : N + 1) {
        if (WALK && kx != (int)(blockIdx.x >> 1))
            __syncthreads();  // the previous column's fold (over sbuf and the stages) has been read
        auto issue = [&](int k) {
            unsigned char *st = stage_base + (size_t)(k & 1) * stage_bytes;
            const ColInput ci = a.ins[w.in_begin + k / 3];
            const FwdSlab sl = a.slabs[ci.slab];
            const int f = k % 3;
            cp_block(st, a.fwd + sl.off + ((size_t)f * (N + 1) + kx) * sl.rows, (size_t)sl.rows * sizeof(C));
            if (spec_quarter(ci.kind)) {
                const T *sp = reinterpret_cast<const T *>(a.spec) + ci.spec_off;
                T *dst = reinterpret_cast<T *>(st + (size_t)N * sizeof(C));
                cp_block(dst, sp + ((size_t)f * (N + 1) + kx) * QS + b * HQ, (size_t)HQ * sizeof(T));
                if (ci.kind == SPEC_QUARTER)
                    cp_block(dst + HQ, sp + ((size_t)(3 + f) * (N + 1) + kx) * QS + b * HQ, (size_t)HQ * sizeof(T));
            } else if constexpr (CS::FULL) {  // this parity's bins ky = 2 k' + b of the x (and y) rows
                const C *sp = reinterpret_cast<const C *>(a.spec) + ci.spec_off;
                const C *rx = sp + ((size_t)f * (N + 1) + kx) * P, *ry = sp + ((size_t)(3 + f) * (N + 1) + kx) * P;
                C *dst = reinterpret_cast<C *>(st + (size_t)N * sizeof(C));
                const bool two = ci.kind == SPEC_FULL;
                for (int q = threadIdx.x; q < N; q += blockDim.x) {
                    cp8(dst + q, rx + 2 * q + b);
                    if (two)
                        cp8(dst + N + q, ry + 2 * q + b);
                }
            }
        };
        issue(0);
        cp_commit();
        if (nitems > 1)
            issue(1);
        cp_commit();

        C acc[2][16];
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            acc[0][u] = hmk<C>(T(0), T(0));
            acc[1][u] = hmk<C>(T(0), T(0));
        }
        for (int k = 0; k < nitems; ++k) {
            cp_wait<1>();
            __syncthreads();
            const unsigned char *st = stage_base + (size_t)(k & 1) * stage_bytes;
            const C *col = reinterpret_cast<const C *>(st);
            const T *spx = reinterpret_cast<const T *>(st + (size_t)N * sizeof(C));
            const ColInput ci = a.ins[w.in_begin + k / 3];
            const int rows = a.slabs[ci.slab].rows;
            const int f = k % 3;
            C v[1][16];
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
                    v[0][u] = x;
                }
            }
            fft_ct<C, false, LOGN, 1, TC>(v, sbuf, SPC, j, active, tw, &tcx);
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
                        C tx = hmk<C>(rx * v[0][u].x, rx * v[0][u].y), ty = hmk<C>(ry * v[0][u].x, ry * v[0][u].y);
                        if (f == 0) {
                            tx = hmk<C>(-tx.y, tx.x);
                            ty = hmk<C>(-ty.y, ty.x);
                        }
                        acc[0][u] = hadd(acc[0][u], tx);
                        acc[1][u] = hadd(acc[1][u], ty);
                    }
                } else if (ci.kind == SPEC_QUARTER_PHI) {
                    // the potential alone: P0 real, Px Py imaginary; mirror signs + P0 Px, - Py
                    const T mx = (f == 2) ? T(-1) : T(1);
#pragma unroll
                    for (int u = 0; u < 16; ++u) {
                        const int kp = j + u * Q;
                        const bool hi = 2 * kp + b > N;
                        const int q = hi ? N - kp - b : kp;
                        const T rx = spx[q] * (hi ? mx : T(1));
                        C tx = hmk<C>(rx * v[0][u].x, rx * v[0][u].y);
                        if (f != 0)
                            tx = hmk<C>(-tx.y, tx.x);
                        acc[0][u] = hadd(acc[0][u], tx);
                    }
                } else if constexpr (CS::FULL) {  // the staged bins of this parity
                    const C *sx = reinterpret_cast<const C *>(st + (size_t)N * sizeof(C)), *sy = sx + N;
                    if (ci.kind == SPEC_FULL_PHI) {
#pragma unroll
                        for (int u = 0; u < 16; ++u)
                            acc[0][u] = hadd(acc[0][u], hmul(sx[j + u * Q], v[0][u]));
                    } else {
#pragma unroll
                        for (int u = 0; u < 16; ++u) {
                            acc[0][u] = hadd(acc[0][u], hmul(sx[j + u * Q], v[0][u]));
                            acc[1][u] = hadd(acc[1][u], hmul(sy[j + u * Q], v[0][u]));
                        }
                    }
                } else if (ci.kind == SPEC_FULL_PHI) {
                    const C *sx = reinterpret_cast<const C *>(a.spec) + ci.spec_off + ((size_t)f * (N + 1) + kx) * P;
#pragma unroll
                    for (int u = 0; u < 16; ++u) {
                        const int ky = 2 * (j + u * Q) + b;
                        acc[0][u] = hadd(acc[0][u], hmul(__ldg(sx + ky), v[0][u]));
                    }
                } else {
                    const C *sx = reinterpret_cast<const C *>(a.spec) + ci.spec_off + ((size_t)f * (N + 1) + kx) * P;
                    const C *sy = reinterpret_cast<const C *>(a.spec) + ci.spec_off + ((size_t)(3 + f) * (N + 1) + kx) * P;
#pragma unroll
                    for (int u = 0; u < 16; ++u) {
                        const int ky = 2 * (j + u * Q) + b;
                        acc[0][u] = hadd(acc[0][u], hmul(__ldg(sx + ky), v[0][u]));
                        acc[1][u] = hadd(acc[1][u], hmul(__ldg(sy + ky), v[0][u]));
                    }
                }
            }
            __syncthreads();  // stage (k & 1) consumed by every thread
            if (k + 2 < nitems)
                issue(k + 2);
            cp_commit();
        }
        cp_wait<0>();
        if (w.slot >= 0) {  // one chunk of a long input list: hand the accumulators to k_col_sum
            if (active) {
#pragma unroll
                for (int comp = 0; comp < 2; ++comp) {
                    C *dst = a.partial + ((((size_t)w.slot * 2 + b) * 2 + comp) * (N + 1) + kx) * N;
#pragma unroll
                    for (int u = 0; u < 16; ++u)
                        dst[j + u * Q] = acc[comp][u];
                }
            }
            continue;  // both CTAs of the cluster take this branch (w is per cluster)
        }
        // inverse column transforms of Fx^ and Fy^ together (the potential: its one
        // component alone); y[n] = even[n] + W_P^{-n} odd[n]
        const bool two = a.ncomp == 2;
        if (two)
            fft_ct<C, true, LOGN, 2, TC>(acc, sbuf, SPC, j, active, tw, &tcx);
        else
            fft_ct<C, true, LOGN, 1, TC>(acc, sbuf, SPC, j, active, tw, &tcx);
        C *fold = sbuf;  // 2N complex over sbuf and the stages
        cluster.sync();
        if (b == 1 && active) {
            C *dst = cluster.map_shared_rank(fold, 0);
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int n = j + u * Q;
                const C w = twist(tw, tl, j, u);
                dst[n] = hmulc(acc[0][u], w);
                if (two)
                    dst[N + n] = hmulc(acc[1][u], w);
            }
        }
        cluster.sync();
        if (b == 0 && active) {
            C *dst = a.bwd + o.off;
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int n = j + u * Q;
                if (n < o.rows) {
                    dst[bwd_index(N, o.rows, 0, kx, n)] = hadd(acc[0][u], fold[n]);
                    if (two)
                        dst[bwd_index(N, o.rows, 1, kx, n)] = hadd(acc[1][u], fold[N + n]);
                }
            }
        }
    }
    if constexpr (TC)
        tc_end(tcx, TCT);
}

// ------------------------------------------------------------------- col_w
// Bytes of one k_col_w input stage: the column, then either the quarter
// spectrum half rows or, for N <= 2048, the full complex spectrum rows of an
// input of Cases 2 and 3 (x and y tables, 2N bins each), so that those are
// copied in ahead like the column instead of being loaded in the product (two
// CTAs per SM still fit at N = 1024, one at 2048, where it measured faster all
// the same; at 4096 two stages would not fit).
template <typename T, int LOGN>
struct ColWStage {
    using C = typename Cx<T>::C;
    static constexpr int N = 1 << LOGN;
    static constexpr bool FULL = LOGN <= 11;
    static constexpr size_t QB = 4 * (size_t)quarter_half(N) * sizeof(T);
    static constexpr size_t FB = FULL ? 2 * (size_t)(2 * N) * sizeof(C) : 0;
    static constexpr size_t BYTES = (size_t)N * sizeof(C) + (QB > FB ? QB : FB);
};

// k_col with both parity halves of a column in one CTA (thread t: half t / Q,
// slot t mod Q), each half's transforms on its own named barrier: every input
// column is staged once for both halves, and 16 warps fit per SM where the
// 2-CTA cluster kernel fits 8 at N = 4096.  Items (input, field) are
// double-buffered as in k_col; a chunk work item hands its accumulators to
// k_col_sum, the others fold the odd half through shared memory, each half
// storing one component.  FP32 without tensor-core tiles, N >= 512 (FP64's two
// sequences per thread need more than 128 registers).
// Batches launch the map rows along x and the columns along y, so that the
// CTAs of one column run the map rows in order: the batch orders its rows so
// that work items reading the same spectra (plans sharing them) are
// neighbours, and those CTAs find the spectrum rows in L2.
// Shared memory: twiddle area | sbuf[2][SPC] | stage[2] { column[N] (complex),
// both halves' two spectrum half rows, [half][x, y][N/2 + 4] reals, or (see
// ColWStage) the full rows [x, y][2N] complex }.  The dual
// inverse transforms of half b use 2 SPC from sbuf + 2 b SPC (reaching over the
// stages, free by then), and the fold reuses the start.
template <typename T, int LOGN, bool BATCH>
__global__ void __launch_bounds__(KShape<LOGN>::ROW_THREADS, 1) k_col_w(SolveArgs<T> a0, BatchView<T> bv)
{
    const int2 wm = BATCH ? bv.map[blockIdx.x] : make_int2(0, (int)blockIdx.y);
    const SolveArgs<T> &a = BATCH ? bv.args[wm.x] : a0;
    using C = typename Cx<T>::C;
    using K = KShape<LOGN>;
    constexpr int N = K::N, Q = K::Q, P = 2 * N, QS = quarter_stride(N), HQ = quarter_half(N);
    constexpr int SPC = col_sp<C>(N);
    constexpr int HB = K::HB_ROW;
    static_assert(HB > 0, "whole warps per half: N >= 512");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *tw = reinterpret_cast<C *>(smem_raw);
    C *sbuf = reinterpret_cast<C *>(smem_raw + tw_bytes<C>(a.tw_entries));
    unsigned char *stage_base = reinterpret_cast<unsigned char *>(sbuf + 2 * SPC);
    using CS = ColWStage<T, LOGN>;
    constexpr size_t stage_bytes = CS::BYTES;
    const int kx = BATCH ? (int)blockIdx.y : (int)blockIdx.x;
    const ColWork w = a.col_list[wm.y];
    const ColOutput o = a.outs[w.out];
    const int t = threadIdx.x;
    const int b = t / Q, j = t - b * Q;
    const int nitems = 3 * w.in_count;
    const TwLayout tl = tw_layout(F16<LOGN>::twlen, N);

    auto issue = [&](int k) {
        unsigned char *st = stage_base + (size_t)(k & 1) * stage_bytes;
        const ColInput ci = a.ins[w.in_begin + k / 3];
        const FwdSlab sl = a.slabs[ci.slab];
        const int f = k % 3;
        cp_block(st, a.fwd + sl.off + ((size_t)f * (N + 1) + kx) * sl.rows, (size_t)sl.rows * sizeof(C));
        if (spec_quarter(ci.kind)) {
            const T *sp = reinterpret_cast<const T *>(a.spec) + ci.spec_off;
            T *dst = reinterpret_cast<T *>(st + (size_t)N * sizeof(C));
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                cp_block(dst + 2 * h * HQ, sp + ((size_t)f * (N + 1) + kx) * QS + h * HQ, (size_t)HQ * sizeof(T));
                if (ci.kind == SPEC_QUARTER)
                    cp_block(dst + (2 * h + 1) * HQ, sp + ((size_t)(3 + f) * (N + 1) + kx) * QS + h * HQ,
                             (size_t)HQ * sizeof(T));
            }
        } else if constexpr (CS::FULL) {  // x (and, forces, y) rows of the full spectra
            const C *sp = reinterpret_cast<const C *>(a.spec) + ci.spec_off;
            C *dst = reinterpret_cast<C *>(st + (size_t)N * sizeof(C));
            cp_block(dst, sp + ((size_t)f * (N + 1) + kx) * P, (size_t)P * sizeof(C));
            if (ci.kind == SPEC_FULL)
                cp_block(dst + P, sp + ((size_t)(3 + f) * (N + 1) + kx) * P, (size_t)P * sizeof(C));
        }
    };
    cp_block(tw, a.tw, tw_bytes<C>(a.tw_entries));
    issue(0);
    cp_commit();
    if (nitems > 1)
        issue(1);
    cp_commit();

    C acc[2][16];
#pragma unroll
    for (int u = 0; u < 16; ++u) {
        acc[0][u] = hmk<C>(T(0), T(0));
        acc[1][u] = hmk<C>(T(0), T(0));
    }
    for (int k = 0; k < nitems; ++k) {
        cp_wait<1>();
        __syncthreads();
        const unsigned char *st = stage_base + (size_t)(k & 1) * stage_bytes;
        const C *col = reinterpret_cast<const C *>(st);
        const T *spx = reinterpret_cast<const T *>(st + (size_t)N * sizeof(C)) + 2 * b * HQ;  // x row; y at + HQ
        const ColInput ci = a.ins[w.in_begin + k / 3];
        const int rows = a.slabs[ci.slab].rows;
        const int f = k % 3;
        C v[1][16];
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const int n = j + u * Q;
            C x = hmk<C>(T(0), T(0));
            if (n < rows) {
                x = col[n];
                if (b)
                    x = hmul(x, twist(tw, tl, j, u));
            }
            v[0][u] = x;
        }
        fft_ct<C, false, LOGN, 1, false, HB>(v, sbuf + b * SPC, SPC, j, true, tw, nullptr, b);
        if (ci.kind == SPEC_QUARTER) {
            // K0x, K0y imaginary (stored Im), the rest real; bins above N read the
            // quarter at P - ky with the table's ky parity: + K0x Kxx Kyy, - Kxy K0y Kyx
            const T mx = (f == 2) ? T(-1) : T(1);
            const T my = (f == 2) ? T(1) : T(-1);
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int kp = j + u * Q;
                const bool hi = 2 * kp + b > N;
                const int q = hi ? N - kp - b : kp;
                const T rx = spx[q] * (hi ? mx : T(1));
                const T ry = spx[HQ + q] * (hi ? my : T(1));
                C tx = hmk<C>(rx * v[0][u].x, rx * v[0][u].y), ty = hmk<C>(ry * v[0][u].x, ry * v[0][u].y);
                if (f == 0) {
                    tx = hmk<C>(-tx.y, tx.x);
                    ty = hmk<C>(-ty.y, ty.x);
                }
                acc[0][u] = hadd(acc[0][u], tx);
                acc[1][u] = hadd(acc[1][u], ty);
            }
        } else if (ci.kind == SPEC_QUARTER_PHI) {
            // the potential alone: P0 real, Px Py imaginary; mirror signs + P0 Px, - Py
            const T mx = (f == 2) ? T(-1) : T(1);
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int kp = j + u * Q;
                const bool hi = 2 * kp + b > N;
                const int q = hi ? N - kp - b : kp;
                const T rx = spx[q] * (hi ? mx : T(1));
                C tx = hmk<C>(rx * v[0][u].x, rx * v[0][u].y);
                if (f != 0)
                    tx = hmk<C>(-tx.y, tx.x);
                acc[0][u] = hadd(acc[0][u], tx);
            }
        } else if constexpr (CS::FULL) {  // the staged full rows
            const C *sx = reinterpret_cast<const C *>(st + (size_t)N * sizeof(C)), *sy = sx + P;
            if (ci.kind == SPEC_FULL_PHI) {
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    const int ky = 2 * (j + u * Q) + b;
                    acc[0][u] = hadd(acc[0][u], hmul(sx[ky], v[0][u]));
                }
            } else {
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    const int ky = 2 * (j + u * Q) + b;
                    acc[0][u] = hadd(acc[0][u], hmul(sx[ky], v[0][u]));
                    acc[1][u] = hadd(acc[1][u], hmul(sy[ky], v[0][u]));
                }
            }
        } else if (ci.kind == SPEC_FULL_PHI) {
            const C *sx = reinterpret_cast<const C *>(a.spec) + ci.spec_off + ((size_t)f * (N + 1) + kx) * P;
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int ky = 2 * (j + u * Q) + b;
                acc[0][u] = hadd(acc[0][u], hmul(__ldg(sx + ky), v[0][u]));
            }
        } else {
            const C *sx = reinterpret_cast<const C *>(a.spec) + ci.spec_off + ((size_t)f * (N + 1) + kx) * P;
            const C *sy = reinterpret_cast<const C *>(a.spec) + ci.spec_off + ((size_t)(3 + f) * (N + 1) + kx) * P;
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int ky = 2 * (j + u * Q) + b;
                acc[0][u] = hadd(acc[0][u], hmul(__ldg(sx + ky), v[0][u]));
                acc[1][u] = hadd(acc[1][u], hmul(__ldg(sy + ky), v[0][u]));
            }
        }
        __syncthreads();  // stage (k & 1) and both exchange buffers consumed by every thread
        if (k + 2 < nitems)
            issue(k + 2);
        cp_commit();
    }
    cp_wait<0>();
    if (w.slot >= 0) {  // one chunk of a long input list: hand the accumulators to k_col_sum
#pragma unroll
        for (int comp = 0; comp < 2; ++comp) {
            C *dst = a.partial + ((((size_t)w.slot * 2 + b) * 2 + comp) * (N + 1) + kx) * N;
#pragma unroll
            for (int u = 0; u < 16; ++u)
                dst[j + u * Q] = acc[comp][u];
        }
        return;
    }
    // both inverse transforms of this half (the potential: its one component
    // alone); y[n] = even[n] + W_P^{-n} odd[n]
    const bool two = a.ncomp == 2;
    if (two)
        fft_ct<C, true, LOGN, 2, false, HB>(acc, sbuf + 2 * b * SPC, SPC, j, true, tw, nullptr, b);
    else
        fft_ct<C, true, LOGN, 1, false, HB>(acc, sbuf + 2 * b * SPC, SPC, j, true, tw, nullptr, b);
    __syncthreads();  // every exchange buffer has been read
    C *fold = sbuf;  // the odd half hands over Fx's twisted values, the even half Fy's own
#pragma unroll
    for (int u = 0; u < 16; ++u) {
        const int n = j + u * Q;
        if (b == 1)
            fold[n] = hmulc(acc[0][u], twist(tw, tl, j, u));
        else if (two)
            fold[N + n] = acc[1][u];
    }
    __syncthreads();
    C *dst = a.bwd + o.off;
#pragma unroll
    for (int u = 0; u < 16; ++u) {
        const int n = j + u * Q;
        if (n >= o.rows)
            continue;
        if (b == 0)
            dst[bwd_index(N, o.rows, 0, kx, n)] = hadd(acc[0][u], fold[n]);
        else if (two)
            dst[bwd_index(N, o.rows, 1, kx, n)] = hadd(fold[N + n], hmulc(acc[1][u], twist(tw, tl, j, u)));
    }
}

// ------------------------------------------------------------------- col_g
// Column pass of a group of Case-3 phase outputs (Sec. 2.2, Eq. eqnbnmn): the
// m^2 outputs of one (coarser source, target) pair convolve the same source
// level with different phase kernels.  One 2-CTA cluster per (column, group):
// the three fields of the source column are transformed once (this parity
// half) and kept in shared memory; then, per output, the spectral
// multiply-accumulate with that phase's spectra and the two inverse transforms,
// together (two sequences per thread), folded through distributed shared
// memory.  Shared memory: twiddle area | sbuf[2 SPC] (the two exchange buffers,
// then the 2N fold) | fld[3][N].
template <typename T, int LOGN, bool BATCH, bool TC>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(KShape<LOGN>::COL_THREADS) k_col_g(SolveArgs<T> a0, BatchView<T> bv)
{
    const int2 wm = BATCH ? bv.map[blockIdx.y] : make_int2(0, (int)blockIdx.y);
    const SolveArgs<T> &a = BATCH ? bv.args[wm.x] : a0;
    using C = typename Cx<T>::C;
    using K = KShape<LOGN>;
    constexpr int N = K::N, Q = K::Q, P = 2 * N;
    constexpr int SPC = col_sp<C>(N);
    extern __shared__ __align__(16) unsigned char smem_tc[];
    constexpr int TCT = tc_tiles(KShape<LOGN>::COL_THREADS, 2);
    constexpr int TCR = tc_round(LOGN, TCT, KK_COL_G);
    static_assert(!TC || sizeof(T) == 4, "tensor-core tiles take FP32 data");
    unsigned char *smem_raw = smem_tc + (TC ? tc_smem_bytes(TCR) : 0);
    TcCtx tcx;
    if constexpr (TC)
        tc_begin(tcx, smem_tc, TCT, TCR, a.status, a.wait_cycles, a.inject);
    C *tw = reinterpret_cast<C *>(smem_raw);
    C *sbuf = reinterpret_cast<C *>(smem_raw + tw_bytes<C>(a.tw_entries));
    C *fld = sbuf + 2 * SPC;  // after the two exchange buffers of the dual inverse
    cg::cluster_group cluster = cg::this_cluster();
    const int b = (int)cluster.block_rank();
    const int kx = blockIdx.x >> 1;
    const int t = threadIdx.x;
    const bool active = t < Q;
    const int j = active ? t : 0;
    const TwLayout tl = tw_layout(F16<LOGN>::twlen, N);
    const ColGroup g = a.groups[wm.y];
    const FwdSlab sl = a.slabs[a.ins[a.outs[g.out_begin].in_begin].slab];
    cp_block(tw, a.tw, tw_bytes<C>(a.tw_entries));
    cp_commit();
    cp_wait<0>();
    __syncthreads();
    C v[1][16];
    for (int f = 0; f < 3; ++f) {
        if (active) {
            const C *col = a.fwd + sl.off + ((size_t)f * (N + 1) + kx) * sl.rows;
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int n = j + u * Q;
                C x = hmk<C>(T(0), T(0));
                if (n < sl.rows) {
                    x = col[n];
                    if (b)
                        x = hmul(x, twist(tw, tl, j, u));
                }
                v[0][u] = x;
            }
        }
        fft_ct<C, false, LOGN, 1, TC>(v, sbuf, SPC, j, active, tw, &tcx);
        if (active) {
#pragma unroll
            for (int u = 0; u < 16; ++u)
                fld[f * N + u * Q + j] = v[0][u];  // read back by this thread only
        }
    }
    const C *spec = reinterpret_cast<const C *>(a.spec);
#pragma unroll 1
    for (int q = 0; q < g.out_count; ++q) {
        const ColOutput o = a.outs[g.out_begin + q];
        const ColInput ci = a.ins[o.in_begin];
        C acc[2][16];
        if (active) {
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                acc[0][u] = hmk<C>(T(0), T(0));
                acc[1][u] = hmk<C>(T(0), T(0));
            }
            if (ci.kind == SPEC_FULL_PHI) {  // the potential alone
#pragma unroll 1
                for (int f = 0; f < 3; ++f) {
                    const C *sx = spec + ci.spec_off + ((size_t)f * (N + 1) + kx) * P;
#pragma unroll
                    for (int u = 0; u < 16; ++u) {
                        const int ky = 2 * (j + u * Q) + b;
                        acc[0][u] = hadd(acc[0][u], hmul(__ldg(sx + ky), fld[f * N + u * Q + j]));
                    }
                }
            } else {
#pragma unroll 1
                for (int f = 0; f < 3; ++f) {
                    const C *sx = spec + ci.spec_off + ((size_t)f * (N + 1) + kx) * P;
                    const C *sy = spec + ci.spec_off + ((size_t)(3 + f) * (N + 1) + kx) * P;
#pragma unroll
                    for (int u = 0; u < 16; ++u) {
                        const int ky = 2 * (j + u * Q) + b;
                        const C x = fld[f * N + u * Q + j];
                        acc[0][u] = hadd(acc[0][u], hmul(__ldg(sx + ky), x));
                        acc[1][u] = hadd(acc[1][u], hmul(__ldg(sy + ky), x));
                    }
                }
            }
        }
        // both inverse transforms together; y[n] = even[n] + W_P^{-n} odd[n]
        fft_ct<C, true, LOGN, 2, TC>(acc, sbuf, SPC, j, active, tw, &tcx);
        cluster.sync();  // both CTAs are done with their exchange buffers
        if (b == 1 && active) {
            C *dst = cluster.map_shared_rank(sbuf, 0);
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const C w = twist(tw, tl, j, u);
                dst[j + u * Q] = hmulc(acc[0][u], w);
                dst[N + j + u * Q] = hmulc(acc[1][u], w);
            }
        }
        cluster.sync();
        if (b == 0 && active) {
            C *out = a.bwd + o.off;
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int n = j + u * Q;
                if (n < o.rows) {
                    out[bwd_index(N, o.rows, 0, kx, n)] = hadd(acc[0][u], sbuf[n]);
                    out[bwd_index(N, o.rows, 1, kx, n)] = hadd(acc[1][u], sbuf[N + n]);
                }
            }
        }
    }
    if constexpr (TC)
        tc_end(tcx, TCT);
}

// ------------------------------------------------------------------ col_gw
// k_col_g with both parity halves in one CTA (thread t: half t / Q, slot t mod
// Q), each half transforming on its own named barrier: half b keeps the three
// transformed source fields at fld + 3 b N, and per output folds through
// shared memory with each half storing one component (the potential: one
// inverse transform, the even half storing).  FP32 without tensor-core tiles,
// 512 <= N <= 2048 (at 4096 the six fields do not fit).
// Shared memory: twiddle area | sbuf[2][2 SPC] (half b's two exchange buffers
// at sbuf + 2 b SPC; the 2N fold at the start) | fld[2][3][N].
template <typename T, int LOGN, bool BATCH>
__global__ void __launch_bounds__(KShape<LOGN>::ROW_THREADS, 1) k_col_gw(SolveArgs<T> a0, BatchView<T> bv)
{
    const int2 wm = BATCH ? bv.map[blockIdx.y] : make_int2(0, (int)blockIdx.y);
    const SolveArgs<T> &a = BATCH ? bv.args[wm.x] : a0;
    using C = typename Cx<T>::C;
    using K = KShape<LOGN>;
    constexpr int N = K::N, Q = K::Q, P = 2 * N;
    constexpr int SPC = col_sp<C>(N);
    constexpr int HB = K::HB_ROW;
    static_assert(HB > 0, "whole warps per half: N >= 512");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *tw = reinterpret_cast<C *>(smem_raw);
    C *sbuf = reinterpret_cast<C *>(smem_raw + tw_bytes<C>(a.tw_entries));
    const int t = threadIdx.x;
    const int b = t / Q, j = t - b * Q;
    C *fld = sbuf + 4 * SPC + 3 * b * N;  // this half's three transformed fields
    const int kx = blockIdx.x;
    const TwLayout tl = tw_layout(F16<LOGN>::twlen, N);
    const ColGroup g = a.groups[wm.y];
    const FwdSlab sl = a.slabs[a.ins[a.outs[g.out_begin].in_begin].slab];
    cp_block(tw, a.tw, tw_bytes<C>(a.tw_entries));
    cp_commit();
    cp_wait<0>();
    __syncthreads();
    {
        C v[1][16];
#pragma unroll 1
        for (int f = 0; f < 3; ++f) {
            const C *col = a.fwd + sl.off + ((size_t)f * (N + 1) + kx) * sl.rows;
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int n = j + u * Q;
                C x = hmk<C>(T(0), T(0));
                if (n < sl.rows) {
                    x = col[n];
                    if (b)
                        x = hmul(x, twist(tw, tl, j, u));
                }
                v[0][u] = x;
            }
            fft_ct<C, false, LOGN, 1, false, HB>(v, sbuf + 2 * b * SPC, SPC, j, true, tw, nullptr, b);
#pragma unroll
            for (int u = 0; u < 16; ++u)
                fld[f * N + u * Q + j] = v[0][u];  // read back by this thread only
        }
    }
    const C *spec = reinterpret_cast<const C *>(a.spec);
    const bool two = a.ncomp == 2;
#pragma unroll 1
    for (int q = 0; q < g.out_count; ++q) {
        const ColOutput o = a.outs[g.out_begin + q];
        const ColInput ci = a.ins[o.in_begin];
        C acc[2][16];
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            acc[0][u] = hmk<C>(T(0), T(0));
            acc[1][u] = hmk<C>(T(0), T(0));
        }
        if (ci.kind == SPEC_FULL_PHI) {  // the potential alone
#pragma unroll 1
            for (int f = 0; f < 3; ++f) {
                const C *sx = spec + ci.spec_off + ((size_t)f * (N + 1) + kx) * P;
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    const int ky = 2 * (j + u * Q) + b;
                    acc[0][u] = hadd(acc[0][u], hmul(__ldg(sx + ky), fld[f * N + u * Q + j]));
                }
            }
        } else {
#pragma unroll 1
            for (int f = 0; f < 3; ++f) {
                const C *sx = spec + ci.spec_off + ((size_t)f * (N + 1) + kx) * P;
                const C *sy = spec + ci.spec_off + ((size_t)(3 + f) * (N + 1) + kx) * P;
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    const int ky = 2 * (j + u * Q) + b;
                    const C x = fld[f * N + u * Q + j];
                    acc[0][u] = hadd(acc[0][u], hmul(__ldg(sx + ky), x));
                    acc[1][u] = hadd(acc[1][u], hmul(__ldg(sy + ky), x));
                }
            }
        }
        // the inverse transforms of this half; y[n] = even[n] + W_P^{-n} odd[n]
        if (two)
            fft_ct<C, true, LOGN, 2, false, HB>(acc, sbuf + 2 * b * SPC, SPC, j, true, tw, nullptr, b);
        else
            fft_ct<C, true, LOGN, 1, false, HB>(acc, sbuf + 2 * b * SPC, SPC, j, true, tw, nullptr, b);
        __syncthreads();  // every exchange buffer has been read
        C *fold = sbuf;
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const int n = j + u * Q;
            if (b == 1)
                fold[n] = hmulc(acc[0][u], twist(tw, tl, j, u));
            else if (two)
                fold[N + n] = acc[1][u];
        }
        __syncthreads();
        C *out = a.bwd + o.off;
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const int n = j + u * Q;
            if (n >= o.rows)
                continue;
            if (b == 0)
                out[bwd_index(N, o.rows, 0, kx, n)] = hadd(acc[0][u], fold[n]);
            else if (two)
                out[bwd_index(N, o.rows, 1, kx, n)] = hadd(fold[N + n], hmulc(acc[1][u], twist(tw, tl, j, u)));
        }
        __syncthreads();  // the fold has been read: the next output's exchanges overwrite it
    }
}

// ----------------------------------------------------------------- col_sum
// Second half of the column pass of an output whose input list was split into
// chunks (k_col work items with a partial slot): the chunks' spectral
// accumulators are summed in slot order, then transformed back and folded as
// in k_col.  Shared memory: twiddle area | two exchange buffers (dual inverse),
// reused for the fold.
template <typename T, int LOGN, bool BATCH, bool TC>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(KShape<LOGN>::COL_THREADS) k_col_sum(SolveArgs<T> a0, BatchView<T> bv)
{
    const int2 wm = BATCH ? bv.map[blockIdx.y] : make_int2(0, (int)blockIdx.y);
    const SolveArgs<T> &a = BATCH ? bv.args[wm.x] : a0;
    using C = typename Cx<T>::C;
    using K = KShape<LOGN>;
    constexpr int N = K::N, Q = K::Q;
    constexpr int SPC = col_sp<C>(N);
    extern __shared__ __align__(16) unsigned char smem_tc[];
    constexpr int TCT = tc_tiles(KShape<LOGN>::COL_THREADS, 2);
    constexpr int TCR = tc_round(LOGN, TCT, KK_COL_SUM);
    static_assert(!TC || sizeof(T) == 4, "tensor-core tiles take FP32 data");
    unsigned char *smem_raw = smem_tc + (TC ? tc_smem_bytes(TCR) : 0);
    TcCtx tcx;
    if constexpr (TC)
        tc_begin(tcx, smem_tc, TCT, TCR, a.status, a.wait_cycles, a.inject);
    C *tw = reinterpret_cast<C *>(smem_raw);
    C *sbuf = reinterpret_cast<C *>(smem_raw + tw_bytes<C>(a.tw_entries));
    cg::cluster_group cluster = cg::this_cluster();
    const int b = (int)cluster.block_rank();
    const int kx = blockIdx.x >> 1;
    const int t = threadIdx.x;
    const bool active = t < Q;
    const int j = active ? t : 0;
    const TwLayout tl = tw_layout(F16<LOGN>::twlen, N);
    const ColSum sm = a.sums[wm.y];
    const ColOutput o = a.outs[sm.out];
    cp_block(tw, a.tw, tw_bytes<C>(a.tw_entries));
    cp_commit();
    C acc[2][16];
#pragma unroll
    for (int u = 0; u < 16; ++u) {
        acc[0][u] = hmk<C>(T(0), T(0));
        acc[1][u] = hmk<C>(T(0), T(0));
    }
    if (active) {
#pragma unroll 1
        for (int k = 0; k < sm.slot_count; ++k) {
#pragma unroll
            for (int comp = 0; comp < 2; ++comp) {
                const C *src = a.partial + ((((size_t)(sm.slot_begin + k) * 2 + b) * 2 + comp) * (N + 1) + kx) * N;
#pragma unroll
                for (int u = 0; u < 16; ++u)
                    acc[comp][u] = hadd(acc[comp][u], src[j + u * Q]);
            }
        }
    }
    cp_wait<0>();
    __syncthreads();
    fft_ct<C, true, LOGN, 2, TC>(acc, sbuf, SPC, j, active, tw, &tcx);
    C *fold = sbuf;
    cluster.sync();
    if (b == 1 && active) {
        C *dst = cluster.map_shared_rank(fold, 0);
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const int n = j + u * Q;
            const C tw_n = twist(tw, tl, j, u);
            dst[n] = hmulc(acc[0][u], tw_n);
            dst[N + n] = hmulc(acc[1][u], tw_n);
        }
    }
    cluster.sync();
    if (b == 0 && active) {
        C *dst = a.bwd + o.off;
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const int n = j + u * Q;
            if (n < o.rows) {
                dst[bwd_index(N, o.rows, 0, kx, n)] = hadd(acc[0][u], fold[n]);
                dst[bwd_index(N, o.rows, 1, kx, n)] = hadd(acc[1][u], fold[N + n]);
            }
        }
    }
    if constexpr (TC)
        tc_end(tcx, TCT);
}

// ------------------------------------------------------------------ row_inv
// Shared memory: twiddle area | stage[N + 1][2 rows] | sbuf[2 SP_ROW] | O[2 comps][2 rows][N].
// The two rows of every (contribution, component) are gathered with
// asynchronous copies -- 16 bytes per bin when both rows are adjacent rows of
// one output, 8 bytes otherwise -- and the next gather is issued as soon as
// the current one has been read into registers, so it overlaps the transform.
template <typename T, int LOGN, bool BATCH, bool TC>
__global__ void __launch_bounds__(KShape<LOGN>::ROW_THREADS) k_row_inv(SolveArgs<T> a0, BatchView<T> bv)
{
    const int2 wm = BATCH ? bv.map[blockIdx.y] : make_int2(0, (int)blockIdx.y);
    const SolveArgs<T> &a = BATCH ? bv.args[wm.x] : a0;
    using C = typename Cx<T>::C;
    using K = KShape<LOGN>;
    constexpr int N = K::N, Q = K::Q, SP = K::SP_ROW, P = 2 * N;
    extern __shared__ __align__(16) unsigned char smem_tc[];
    constexpr int TCT = tc_tiles(KShape<LOGN>::ROW_THREADS, 1);
    constexpr int TCR = tc_round(LOGN, TCT, KK_ROW_INV);
    static_assert(!TC || sizeof(T) == 4, "tensor-core tiles take FP32 data");
    unsigned char *smem_raw = smem_tc + (TC ? tc_smem_bytes(TCR) : 0);
    TcCtx tcx;
    if constexpr (TC)
        tc_begin(tcx, smem_tc, TCT, TCR, a.status, a.wait_cycles, a.inject);
    C *tw = reinterpret_cast<C *>(smem_raw);
    C *stg = reinterpret_cast<C *>(smem_raw + tw_bytes<C>(a.tw_entries));  // [kx][2]
    C *sbuf = stg + 2 * (N + 1) + ((2 * (N + 1) * sizeof(C)) % 16 ? 1 : 0);
    T *O = reinterpret_cast<T *>(sbuf + 2 * SP);
    const int tl = BATCH ? wm.y : a.level_base + wm.y;
    const int j0 = 2 * blockIdx.x, j1 = j0 + 1;
    const int t = threadIdx.x;
    const bool active = t < 2 * Q;
    const int b = active ? t / Q : 0, j = active ? t - b * Q : 0;
    const TwLayout twl = tw_layout(F16<LOGN>::twlen, N);
    const int c0 = a.contrib_begin[tl], c1 = a.contrib_begin[tl + 1];
    const int nc = a.ncomp;  // 2 (Fx, Fy) or 1 (the potential)
    const int nitems = nc * (c1 - c0);  // (contribution, component)

    auto issue = [&](int k) {
        const RowContrib rc = a.contribs[c0 + (k >> (nc - 1))];
        const int comp = k & (nc - 1);
        const ColOutput oa = a.outs[rc.out_base + (j0 % rc.m) * rc.m];
        const ColOutput ob = a.outs[rc.out_base + (j1 % rc.m) * rc.m];
        const int ra = j0 / rc.m, rb = j1 / rc.m;
        const C *ba = a.bwd + oa.off + bwd_index(N, oa.rows, comp, 0, ra);
        const C *bb = a.bwd + ob.off + bwd_index(N, ob.rows, comp, 0, rb);
        if (rc.m == 1) {  // rows j0, j0 + 1 of one output: one piece per bin
            constexpr int PG = 2 * (int)sizeof(C) / 16;
            for (int q = t; q < (N + 1) * PG; q += K::ROW_THREADS) {
                const int kx = q / PG, piece = q - kx * PG;
                cp16(stg + 2 * kx + piece * (16 / (int)sizeof(C)), ba + (size_t)kx * oa.rows + piece * (16 / (int)sizeof(C)));
            }
        } else {
            for (int q = t; q < 2 * (N + 1); q += K::ROW_THREADS) {
                const int kx = q >> 1, row = q & 1;
                const C *s = row ? bb + (size_t)kx * ob.rows : ba + (size_t)kx * oa.rows;
                if (sizeof(C) == 8)
                    cp8(stg + 2 * kx + row, s);
                else
                    cp16(stg + 2 * kx + row, s);
            }
        }
    };
    cp_block(tw, a.tw, tw_bytes<C>(a.tw_entries));
    if (nitems > 0)
        issue(0);
    cp_commit();
    for (int i = t; i < 4 * N; i += K::ROW_THREADS)
        O[i] = T(0);
    for (int k = 0; k < nitems; ++k) {
        const RowContrib rc = a.contribs[c0 + (k >> (nc - 1))];
        const int comp = k & (nc - 1);
        const int nout = N / rc.m;
        cp_wait<0>();
        __syncthreads();
        C v[1][16];
        if (active) {
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int kx = 2 * (j + u * Q) + b;
                const int k2 = kx <= N ? kx : P - kx;
                const C A = stg[2 * k2], B = stg[2 * k2 + 1];
                // Z = A + iB, from the stored half (kx <= N) or its conjugate mirror
                v[0][u] = kx <= N ? hmk<C>(A.x - B.y, A.y + B.x) : hmk<C>(A.x + B.y, B.x - A.y);
            }
        }
        __syncthreads();  // the stage has been read
        if (k + 1 < nitems)
            issue(k + 1);
        cp_commit();
        // the block barrier above also follows the previous item's fold
        constexpr int HB = TC ? 0 : K::HB_ROW;
        fft_ct<C, true, LOGN, 1, TC, HB>(v, sbuf + b * SP, SP, j, active, tw, &tcx, b);
        __syncthreads();
        if (active && b == 1) {
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int n = j + u * Q;
                sbuf[pad16(n)] = hmulc(v[0][u], twist(tw, twl, j, u));
            }
        }
        __syncthreads();
        if (active && b == 0) {
            T *Oc = O + comp * 2 * N;
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int n = j + u * Q;
                if (n < nout) {
                    const C y = hadd(v[0][u], sbuf[pad16(n)]);
                    const int i = rc.m * n + rc.px;
                    Oc[i] += y.x;
                    Oc[N + i] += y.y;
                }
            }
        }
    }
    __syncthreads();
    T *fx = a.fx[tl], *fy = a.fy[tl];
    for (int i = t; i < N; i += K::ROW_THREADS) {
        const bool ca = covered(a, tl, j0, i), cb = covered(a, tl, j1, i);
        fx[(size_t)j0 * N + i] = ca ? T(0) : O[i];
        fx[(size_t)j1 * N + i] = cb ? T(0) : O[N + i];
        if (nc == 2) {
            fy[(size_t)j0 * N + i] = ca ? T(0) : O[2 * N + i];
            fy[(size_t)j1 * N + i] = cb ? T(0) : O[3 * N + i];
        }
    }
    if constexpr (TC)
        tc_end(tcx, TCT);
}

// ----------------------------------------------------------------- row_inv1
// Inverse row pass of a patch with a single contribution, its own main output
// (m = 1: the level-0 patches, every uniform solve).  NC = 1: one CTA per
// (row pair, component); NC = 2: one CTA per row pair, a thread carrying the
// same slot of both components (two sequences sharing the barriers).  The two
// rows of a component are gathered (16 bytes per bin in FP32), turned into one
// complex sequence Z = A + iB by the Hermitian extension, inverse transformed as
// two parity halves, folded, and stored straight from registers.  The exchange
// buffer of the transform aliases the gather stage.
// Grid: x = component * N/2 + row pair (NC = 1; component 0 only for the
// potential) or row pair (NC = 2), y = work item (batch) or patch from level_base.
// The tensor-core instances are launched with fewer CTAs in x (the resident
// CTAs shared among the patches), each walking those items in turn.
template <typename T, int LOGN, bool BATCH, bool TC, int NC>
__global__ void __launch_bounds__(KShape<LOGN>::ROW_THREADS, sizeof(T) == 4 && !TC && NC == 1 ? 2 : 1)
    k_row_inv1(SolveArgs<T> a0, BatchView<T> bv)
{
    const int2 wm = BATCH ? bv.map[blockIdx.y] : make_int2(0, (int)blockIdx.y);
    const SolveArgs<T> &a = BATCH ? bv.args[wm.x] : a0;
    using C = typename Cx<T>::C;
    using K = KShape<LOGN>;
    constexpr int N = K::N, Q = K::Q, SP = K::SP_ROW, P = 2 * N;
    extern __shared__ __align__(16) unsigned char smem_tc[];
    constexpr int TCT = tc_tiles(KShape<LOGN>::ROW_THREADS, NC);
    constexpr int TCR = tc_round(LOGN, TCT, NC == 1 ? KK_ROW_INV1 : KK_ROW_INV2);
    static_assert(!TC || sizeof(T) == 4, "tensor-core tiles take FP32 data");
    unsigned char *smem_raw = smem_tc + (TC ? tc_smem_bytes(TCR) : 0);
    TcCtx tcx;
    if constexpr (TC)
        tc_begin(tcx, smem_tc, TCT, TCR, a.status, a.wait_cycles, a.inject);
    C *tw = reinterpret_cast<C *>(smem_raw);
    // stage: component c, bin kx's two rows (a pair of C) at [c][kx & 1][kx >> 1], so
    // the threads of a parity half read consecutive pairs; then the exchange buffers
    C *stg = reinterpret_cast<C *>(smem_raw + tw_bytes<C>(a.tw_entries));
    constexpr int HALF = N / 2 + 1;
    C *sbuf = stg;
    const int tl = BATCH ? wm.y : a.level_base + wm.y;
    const int t = threadIdx.x;
    const bool active = t < 2 * Q;
    const int b = active ? t / Q : 0, j = active ? t - b * Q : 0;
    const TwLayout twl = tw_layout(F16<LOGN>::twlen, N);
    const RowContrib rc = a.contribs[a.contrib_begin[tl]];
    const ColOutput o = a.outs[rc.out_base];
    cp_block(tw, a.tw, tw_bytes<C>(a.tw_entries));
    // tensor-core instances walk the grid's x items (tiles and tensor memory set up once per CTA)
    constexpr bool WALK = TC && !BATCH;
    const int items = WALK ? (NC == 1 ? a.ncomp : 1) * (N / 2) : (int)gridDim.x;
    for (int it = blockIdx.x; it < items; it += gridDim.x) {
        if (WALK && it != (int)blockIdx.x)
            __syncthreads();  // the previous item's stores have read the exchange buffers
        const int comp0 = NC == 1 && it >= N / 2 ? 1 : 0;
        const int j0 = 2 * (it - comp0 * (N / 2)), j1 = j0 + 1;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const C *base = a.bwd + o.off + bwd_index(N, o.rows, comp0 + c, 0, j0);
            constexpr int PG = 2 * (int)sizeof(C) / 16;  // 16-byte pieces per bin (rows j0, j1 adjacent)
            for (int q = t; q < (N + 1) * PG; q += K::ROW_THREADS) {
                const int kx = q / PG, piece = q - kx * PG;
                C *dst = stg + 2 * ((c * 2 + (kx & 1)) * HALF + (kx >> 1));
                cp16(dst + piece * (16 / (int)sizeof(C)), base + (size_t)kx * o.rows + piece * (16 / (int)sizeof(C)));
            }
        }
        cp_commit();
        cp_wait<0>();
        __syncthreads();
        C v[NC][16];
        if (active) {
#pragma unroll
            for (int c = 0; c < NC; ++c)
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    const int kx = 2 * (j + u * Q) + b;
                    const int k2 = kx <= N ? kx : P - kx;  // same parity as kx
                    const C *pr = stg + 2 * ((c * 2 + b) * HALF + (k2 >> 1));
                    C A, B;
                    if constexpr (sizeof(T) == 4) {  // one 16-byte load (pairs start on 16-byte boundaries)
                        const float4 ab = *reinterpret_cast<const float4 *>(pr);
                        A = hmk<C>(ab.x, ab.y);
                        B = hmk<C>(ab.z, ab.w);
                    } else {
                        A = pr[0];
                        B = pr[1];
                    }
                    v[c][u] = kx <= N ? hmk<C>(A.x - B.y, A.y + B.x) : hmk<C>(A.x + B.y, B.x - A.y);
                }
        }
        // the transform's first exchange write follows a barrier, after every read of the stage;
        // half b's NC sequences at sbuf + (b NC + c) SP
        constexpr int HB = TC ? 0 : K::HB_ROW;
        if constexpr (HB > 0)
            __syncthreads();  // half 0's exchange buffer overlaps half 1's part of the stage
        fft_ct<C, true, LOGN, NC, TC, HB>(v, sbuf + b * NC * SP, SP, j, active, tw, &tcx, b);
        __syncthreads();
        if (active && b == 1) {
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int n = j + u * Q;
                const C w = twist(tw, twl, j, u);
#pragma unroll
                for (int c = 0; c < NC; ++c)
                    sbuf[c * SP + pad16(n)] = hmulc(v[c][u], w);
            }
        }
        __syncthreads();
        if (active && b == 0) {
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                T *out = comp0 + c ? a.fy[tl] : a.fx[tl];
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    const int n = j + u * Q;
                    const C y = hadd(v[c][u], sbuf[c * SP + pad16(n)]);
                    out[(size_t)j0 * N + n] = covered(a, tl, j0, n) ? T(0) : y.x;
                    out[(size_t)j1 * N + n] = covered(a, tl, j1, n) ? T(0) : y.y;
                }
            }
        }
        if (!WALK)
            break;
    }
    if constexpr (TC)
        tc_end(tcx, TCT);
}

// ---------------------------------------------------------------- row_inv1t
// k_row_inv1 (one CTA per row pair and component) with the gather done by the
// tensor memory accelerator: the level-0 main column output, seen as a 2-D
// tensor of floats [comp * (N+1) + kx][2N] (a.tmap_inv, encoded at plan
// creation), is copied in boxes of kTmaBox bins x one row pair (16 bytes a bin)
// into shared memory in bin order.  One thread issues the copies; every thread
// waits on an mbarrier (bounded: a timeout sets STATUS_TMA_TIMEOUT).  The rest
// is k_row_inv1's: Hermitian extension, two parity halves (half barriers), fold.
// Shared memory: 128-byte aligned stage (aliased by the exchange buffers) |
// twiddle area | mbarrier.  FP32, N >= 512, no batch view.
constexpr long long kTmaWaitCycles = 2000000000LL;  // about one second at the SM clock

template <typename T, int LOGN>
__host__ __device__ constexpr size_t row_inv1t_body()
{
    using C = typename Cx<T>::C;
    constexpr int N = 1 << LOGN;
    constexpr size_t stage = (size_t)((N + 1 + kTmaBox - 1) / kTmaBox) * kTmaBox * 16;
    constexpr size_t xbuf = 2 * (size_t)KShape<LOGN>::SP_ROW * sizeof(C);
    return ((stage > xbuf ? stage : xbuf) + 127) & ~(size_t)127;
}

template <typename T, int LOGN>
__global__ void __launch_bounds__(KShape<LOGN>::ROW_THREADS, 2) k_row_inv1t(const __grid_constant__ SolveArgs<T> a)
{
    static_assert(sizeof(T) == 4 && KShape<LOGN>::HB_ROW > 0, "FP32, N >= 512");
    using C = typename Cx<T>::C;
    using K = KShape<LOGN>;
    constexpr int N = K::N, Q = K::Q, SP = K::SP_ROW, P = 2 * N;
    constexpr int NBOX = (N + 1 + kTmaBox - 1) / kTmaBox;
    constexpr uint32_t STAGE_BYTES = (uint32_t)NBOX * kTmaBox * 16;
    constexpr size_t BODY = row_inv1t_body<T, LOGN>();
    extern __shared__ __align__(16) unsigned char smem_dyn[];
    // the copies want a 128-byte aligned destination: the launch adds 128 bytes of slack
    const uint32_t base_s = (uint32_t)__cvta_generic_to_shared(smem_dyn);
    unsigned char *smem_raw = smem_dyn + (((base_s + 127u) & ~127u) - base_s);
    unsigned char *stage = smem_raw;
    C *sbuf = reinterpret_cast<C *>(smem_raw);
    C *tw = reinterpret_cast<C *>(smem_raw + BODY);
    const uint32_t mb = (uint32_t)__cvta_generic_to_shared(smem_raw + BODY + tw_bytes<C>(a.tw_entries));
    const int tl = a.level_base;
    const int comp0 = (int)blockIdx.x >= N / 2 ? 1 : 0;
    const int j0 = 2 * ((int)blockIdx.x - comp0 * (N / 2)), j1 = j0 + 1;
    const int t = threadIdx.x;
    const int b = t / Q, j = t - b * Q;  // every thread holds a slot (2Q threads)
    const TwLayout twl = tw_layout(F16<LOGN>::twlen, N);
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(mb), "r"(1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    cp_block(tw, a.tw, tw_bytes<C>(a.tw_entries));
    cp_commit();
    __syncthreads();  // the mbarrier is initialised
    if (t == 0 && !(a.inject & INJECT_TMA_GATHER)) {  // (a test may withhold the copies)
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mb), "r"(STAGE_BYTES) : "memory");
        const unsigned long long map = reinterpret_cast<unsigned long long>(&a.tmap_inv[0]);
        for (int k = 0; k < NBOX; ++k) {
            const uint32_t dst = (uint32_t)__cvta_generic_to_shared(stage + (size_t)k * kTmaBox * 16);
            const int x = 2 * j0, y = comp0 * (N + 1) + k * kTmaBox;  // x: 4 floats a row pair, 16-byte aligned
            asm volatile(
                "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
                "[%4];\n" ::"r"(dst),
                "l"(map), "r"(x), "r"(y), "r"(mb)
                : "memory");
        }
    }
    cp_wait<0>();
    // bounded wait for the gather; if any thread gave up, the CTA records it, waits once
    // more (bounded) for copies that may still land in its shared memory, and returns
    const long long bound = a.wait_cycles > 0 ? a.wait_cycles : kTmaWaitCycles;
    const bool landed = tc_try_wait(mb, 0u, bound);
    if (__syncthreads_or(!landed)) {
        if (t == 0)
            atomicOr(a.status, STATUS_TMA_TIMEOUT);
        tc_try_wait(mb, 0u, bound);
        return;
    }
    C v[1][16];
#pragma unroll
    for (int u = 0; u < 16; ++u) {
        const int kx = 2 * (j + u * Q) + b;
        const int k2 = kx <= N ? kx : P - kx;
        const float4 ab = *reinterpret_cast<const float4 *>(stage + (size_t)k2 * 16);
        const C A = hmk<C>(ab.x, ab.y), B = hmk<C>(ab.z, ab.w);
        v[0][u] = kx <= N ? hmk<C>(A.x - B.y, A.y + B.x) : hmk<C>(A.x + B.y, B.x - A.y);
    }
    __syncthreads();  // the stage has been read: the exchange buffers alias it
    fft_ct<C, true, LOGN, 1, false, K::HB_ROW>(v, sbuf + b * SP, SP, j, true, tw, nullptr, b);
    __syncthreads();
    // fold y = even + W_P^{-n} odd: the even half stores n < N/2 (slots u < 8), the
    // odd half n >= N/2, each handing the other its values of the other range
#pragma unroll
    for (int u = 0; u < 16; ++u) {
        const int n = j + u * Q;
        if (b == 1 && u < 8)
            sbuf[pad16(n)] = hmulc(v[0][u], twist(tw, twl, j, u));
        else if (b == 0 && u >= 8)
            sbuf[pad16(n)] = v[0][u];
    }
    __syncthreads();
    T *out = comp0 ? a.fy[tl] : a.fx[tl];
#pragma unroll
    for (int u = 0; u < 16; ++u) {
        const int n = j + u * Q;
        if ((b == 0) != (u < 8))
            continue;
        const C y = b == 0 ? hadd(v[0][u], sbuf[pad16(n)]) : hadd(sbuf[pad16(n)], hmulc(v[0][u], twist(tw, twl, j, u)));
        out[(size_t)j0 * N + n] = covered(a, tl, j0, n) ? T(0) : y.x;
        out[(size_t)j1 * N + n] = covered(a, tl, j1, n) ? T(0) : y.y;
    }
}

// ---------------------------------------------------------------- row_inv1x
// The level-0 inverse row pass of k_row_inv1t with the structure of k_col_mx:
// one thread per slot j carries both parity halves of a row pair's inverse
// transform (the fold y = even + W_P^{-n} odd is done in registers) with the
// slot's stage twiddles in registers, and the CTA walks its (row pair,
// component) items: as soon as an item's bins are in registers, the tensor
// memory accelerator gathers the next item's bins into the same stage behind
// the transforms (the exchange buffers do not alias the stage).  G = 256 /
// (N/16) groups of N/16 threads per CTA, each walking its own items on its own
// named barrier and mbarrier.  Waits are bounded: a group that gives up records
// STATUS_TMA_TIMEOUT, waits once more (bounded) for copies still landing in its
// stage, and stops.  FP32, N >= 1024, one level-0 patch, no batch view.
// Shared memory per group: 128-byte aligned stage | exchange buffers
// [2][SP_ROW] | mbarrier, flag.
template <int LOGN>
struct KRx {
    static constexpr int N = 1 << LOGN, Q = N >> 4;
    static constexpr int G = Q >= 256 ? 1 : 256 / Q;
    static constexpr int THREADS = G * Q;
    static constexpr int NBOX = (N + 1 + kTmaBox - 1) / kTmaBox;
    static constexpr uint32_t STAGE_BYTES = (uint32_t)NBOX * kTmaBox * 16;
    static constexpr size_t XB = 2 * (size_t)KShape<LOGN>::SP_ROW * 8;
    static constexpr size_t GROUP_BYTES = ((STAGE_BYTES + XB + 16 + 127) / 128) * 128;
    static constexpr size_t SMEM = G * GROUP_BYTES + 128;  // + alignment slack
};

template <int LOGN, int PLAN>
__global__ void __launch_bounds__(KRx<LOGN>::THREADS, 1) k_row_inv1x(const __grid_constant__ SolveArgs<float> a)
{
    using C = float2;
    using R = KRx<LOGN>;
    using P = FR<LOGN, PLAN>;
    constexpr int N = R::N, Q = R::Q, G = R::G, SP = KShape<LOGN>::SP_ROW, PP = 2 * N;
    static_assert(Q >= 64, "named group barriers need whole warps");
    extern __shared__ __align__(16) unsigned char smem_dyn[];
    const uint32_t base_s = (uint32_t)__cvta_generic_to_shared(smem_dyn);
    unsigned char *smem_al = smem_dyn + (((base_s + 127u) & ~127u) - base_s);
    const int t = threadIdx.x;
    const int g = t / Q, j = t - g * Q;
    unsigned char *gb = smem_al + (size_t)g * R::GROUP_BYTES;
    unsigned char *stage = gb;
    C *xb = reinterpret_cast<C *>(gb + R::STAGE_BYTES);
    const uint32_t mb = (uint32_t)__cvta_generic_to_shared(gb + R::STAGE_BYTES + R::XB);
    volatile int *gave_up = reinterpret_cast<volatile int *>(gb + R::STAGE_BYTES + R::XB + 8);
    const unsigned bar = 1 + g;
    const int tl = a.level_base;
    const int items = a.ncomp * (N / 2);
    C trw[P::NST - 1][15];
    load_twiddles_rt<C, LOGN, PLAN>(trw, a.twn, j);
    const TwLayout twl = tw_layout(F16<LOGN>::twlen, N);
    const C wj = a.tw[twl.base + j];  // W_P^j
    auto twist_u = [&](int u) { return hmul(wj, hmk<C>((float)kW32c[u], (float)-kW32s[u])); };
    const long long bound = a.wait_cycles > 0 ? a.wait_cycles : kTmaWaitCycles;
    const bool withhold = (a.inject & INJECT_TMA_GATHER) != 0;
    auto gather = [&](int it) {  // one thread of the group: the bins of item it
        if (withhold)
            return;  // (a test withholds the copies)
        // the stage was last read through the generic proxy: order that before the copies
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        const int comp = it >= N / 2 ? 1 : 0;
        const int j0 = 2 * (it - comp * (N / 2));
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mb), "r"(R::STAGE_BYTES)
                     : "memory");
        const unsigned long long map = reinterpret_cast<unsigned long long>(&a.tmap_inv[0]);
        for (int k = 0; k < R::NBOX; ++k) {
            const uint32_t dst = (uint32_t)__cvta_generic_to_shared(stage + (size_t)k * kTmaBox * 16);
            const int x = 2 * j0, y = comp * (N + 1) + k * kTmaBox;  // x: 4 floats a row pair, 16-byte aligned
            asm volatile(
                "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
                "[%4];\n" ::"r"(dst),
                "l"(map), "r"(x), "r"(y), "r"(mb)
                : "memory");
        }
    };
    const int step = (int)gridDim.x * G;
    int it = (int)blockIdx.x * G + g;
    if (j == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(mb), "r"(1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        *gave_up = 0;
    }
    group_sync(bar, Q);  // the mbarrier is initialised
    if (j == 0 && it < items)
        gather(it);
    for (uint32_t phase = 0; it < items; it += step, ++phase) {  // uniform over the group
        if (!tc_try_wait(mb, phase & 1u, bound))
            *gave_up = 1;
        group_sync(bar, Q);
        if (*gave_up) {  // every thread of the group sees it after the barrier
            if (j == 0)
                atomicOr(a.status, STATUS_TMA_TIMEOUT);
            tc_try_wait(mb, phase & 1u, bound);  // copies that may still land in the stage
            break;
        }
        const int comp = it >= N / 2 ? 1 : 0;
        const int j0 = 2 * (it - comp * (N / 2)), j1 = j0 + 1;
        C v[2][16];
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int kx = 2 * (j + u * Q) + b;
                const int k2 = kx <= N ? kx : PP - kx;
                const float4 ab = *reinterpret_cast<const float4 *>(stage + (size_t)k2 * 16);
                const C A = hmk<C>(ab.x, ab.y), B = hmk<C>(ab.z, ab.w);
                v[b][u] = kx <= N ? hmk<C>(A.x - B.y, A.y + B.x) : hmk<C>(A.x + B.y, B.x - A.y);
            }
        group_sync(bar, Q);  // every thread has read the stage
        if (j == 0 && it + step < items)
            gather(it + step);
        fft_stages_rt<C, true, LOGN, PLAN, 2, 0>(v, xb, SP, j, trw, bar, Q);
        float *out = comp ? a.fy[tl] : a.fx[tl];
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const int n = j + u * Q;
            const C y = hadd(v[0][u], hmulc(v[1][u], twist_u(u)));
            out[(size_t)j0 * N + n] = covered(a, tl, j0, n) ? 0.0f : y.x;
            out[(size_t)j1 * N + n] = covered(a, tl, j1, n) ? 0.0f : y.y;
        }
    }
}

// ---------------------------------------------------------------- row_inv2x
// k_row_inv1x with two row pairs per item: the tensor memory accelerator gathers
// both pairs' bins of one component at once, so each copied piece is the 32
// bytes of two neighbouring pairs (a.tmap_inv encoded with boxes of 8 floats),
// half the requests a pair-by-pair gather makes.  The two pairs are
// transformed one after the other from the stage; the next item's gather is
// issued once the second pair is in registers.  A thread reads its two parity
// halves' bins in the order (s, 1 - s), s = bit 1 of its slot, so that the eight
// threads of a quarter warp touch eight distinct 16-byte bank groups in pairs
// (two-way, as the one-pair stage) instead of four-way.  G groups as many as fit
// in shared memory (at most 256 threads).  FP32, N >= 1024, one level-0 patch.
// Dynamic shared memory a CTA may opt in to (227 KB).
constexpr size_t kMaxDynSmem = 232448;

template <int LOGN>
struct KR2x {
    static constexpr int N = 1 << LOGN, Q = N >> 4;
    static constexpr int NBOX = (N + 1 + kTmaBox - 1) / kTmaBox;
    static constexpr uint32_t STAGE_BYTES = (uint32_t)NBOX * kTmaBox * 32;
    static constexpr size_t XB = 2 * (size_t)KShape<LOGN>::SP_ROW * 8;
    static constexpr size_t GROUP_BYTES = ((STAGE_BYTES + XB + 16 + 127) / 128) * 128;
    static constexpr int GMAX = Q >= 256 ? 1 : 256 / Q;
    static constexpr int GFIT = (int)((kMaxDynSmem - 128) / GROUP_BYTES);
    static constexpr int G = GFIT < GMAX ? GFIT : GMAX;
    static constexpr int THREADS = G * Q;
    static constexpr size_t SMEM = G * GROUP_BYTES + 128;  // + alignment slack
    static_assert(G >= 1, "one group's stage must fit in shared memory");
};

template <int LOGN, int PLAN>
__global__ void __launch_bounds__(KR2x<LOGN>::THREADS, 1) k_row_inv2x(const __grid_constant__ SolveArgs<float> a)
{
    using C = float2;
    using R = KR2x<LOGN>;
    using P = FR<LOGN, PLAN>;
    constexpr int N = R::N, Q = R::Q, SP = KShape<LOGN>::SP_ROW, PP = 2 * N;
    static_assert(Q >= 64, "named group barriers need whole warps");
    extern __shared__ __align__(16) unsigned char smem_dyn[];
    const uint32_t base_s = (uint32_t)__cvta_generic_to_shared(smem_dyn);
    unsigned char *smem_al = smem_dyn + (((base_s + 127u) & ~127u) - base_s);
    const int t = threadIdx.x;
    const int g = t / Q, j = t - g * Q;
    unsigned char *gb = smem_al + (size_t)g * R::GROUP_BYTES;
    unsigned char *stage = gb;
    C *xb = reinterpret_cast<C *>(gb + R::STAGE_BYTES);
    const uint32_t mb = (uint32_t)__cvta_generic_to_shared(gb + R::STAGE_BYTES + R::XB);
    volatile int *gave_up = reinterpret_cast<volatile int *>(gb + R::STAGE_BYTES + R::XB + 8);
    const unsigned bar = 1 + g;
    const int tl = a.level_base;
    const int items = a.ncomp * (N / 4);
    C trw[P::NST - 1][15];
    load_twiddles_rt<C, LOGN, PLAN>(trw, a.twn, j);
    const TwLayout twl = tw_layout(F16<LOGN>::twlen, N);
    const C wj = a.tw[twl.base + j];  // W_P^j
    auto twist_u = [&](int u) { return hmul(wj, hmk<C>((float)kW32c[u], (float)-kW32s[u])); };
    const long long bound = a.wait_cycles > 0 ? a.wait_cycles : kTmaWaitCycles;
    const bool withhold = (a.inject & INJECT_TMA_GATHER) != 0;
    const int s = (j >> 1) & 1;  // which parity half this thread reads first
    auto gather = [&](int it) {  // one thread of the group: the bins of item it
        if (withhold)
            return;  // (a test withholds the copies)
        // the stage was last read through the generic proxy: order that before the copies
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        const int comp = it >= N / 4 ? 1 : 0;
        const int q = it - comp * (N / 4);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mb), "r"(R::STAGE_BYTES)
                     : "memory");
        const unsigned long long map = reinterpret_cast<unsigned long long>(&a.tmap_inv[0]);
        for (int k = 0; k < R::NBOX; ++k) {
            const uint32_t dst = (uint32_t)__cvta_generic_to_shared(stage + (size_t)k * kTmaBox * 32);
            const int x = 8 * q, y = comp * (N + 1) + k * kTmaBox;  // x: 8 floats two row pairs, 32-byte aligned
            asm volatile(
                "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
                "[%4];\n" ::"r"(dst),
                "l"(map), "r"(x), "r"(y), "r"(mb)
                : "memory");
        }
    };
    // bin kx of pair h (0, 1) of the staged item as the packed complex row value
    auto bin = [&](int kx, int h) {
        const int k2 = kx <= N ? kx : PP - kx;
        const float4 ab = *reinterpret_cast<const float4 *>(stage + (size_t)k2 * 32 + h * 16);
        const C A = hmk<C>(ab.x, ab.y), B = hmk<C>(ab.z, ab.w);
        return kx <= N ? hmk<C>(A.x - B.y, A.y + B.x) : hmk<C>(A.x + B.y, B.x - A.y);
    };
    const int step = (int)gridDim.x * R::G;
    int it = (int)blockIdx.x * R::G + g;
    if (j == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(mb), "r"(1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        *gave_up = 0;
    }
    group_sync(bar, Q);  // the mbarrier is initialised
    if (j == 0 && it < items)
        gather(it);
    for (uint32_t phase = 0; it < items; it += step, ++phase) {  // uniform over the group
        if (!tc_try_wait(mb, phase & 1u, bound))
            *gave_up = 1;
        group_sync(bar, Q);
        if (*gave_up) {  // every thread of the group sees it after the barrier
            if (j == 0)
                atomicOr(a.status, STATUS_TMA_TIMEOUT);
            tc_try_wait(mb, phase & 1u, bound);  // copies that may still land in the stage
            break;
        }
        const int comp = it >= N / 4 ? 1 : 0;
        const int q = it - comp * (N / 4);
        float *out = comp ? a.fy[tl] : a.fx[tl];
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
            C v[2][16];
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int k0 = 2 * (j + u * Q);
                const C first = bin(k0 + s, h), second = bin(k0 + 1 - s, h);
                v[0][u] = s ? second : first;
                v[1][u] = s ? first : second;
            }
            if (h == 1) {
                group_sync(bar, Q);  // every thread has read the stage (and pair 0's exchanges)
                if (j == 0 && it + step < items)
                    gather(it + step);
            }
            fft_stages_rt<C, true, LOGN, PLAN, 2, 0>(v, xb, SP, j, trw, bar, Q);
            const int j0 = 4 * q + 2 * h, j1 = j0 + 1;
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int n = j + u * Q;
                const C y = hadd(v[0][u], hmulc(v[1][u], twist_u(u)));
                out[(size_t)j0 * N + n] = covered(a, tl, j0, n) ? 0.0f : y.x;
                out[(size_t)j1 * N + n] = covered(a, tl, j1, n) ? 0.0f : y.y;
            }
        }
    }
}

// ------------------------------------------------------------ zero-rim path
// Forward row pass of a SGF_PLAN_ZERO_RIM plan: the rows of sigma alone (the
// slopes are folded into the merged spectra).  Also verifies the guarantee:
// the CTAs of rows 0-1 and N-2..N-1 scan their rows, every CTA its cells in
// columns 0, 1, N-2, N-1; a nonzero value sets STATUS_RIM_NONZERO.
// The CTA walks the row pairs blockIdx.x, blockIdx.x + gridDim.x, ...: once a
// pair's rows are in registers, the next pair's rows are copied in behind the
// transform.  Only the tensor-core instances walk (launched with the CTAs that
// fit at once; each CTA builds its DFT tiles and takes its tensor memory once);
// the others, and batches, take one row pair per CTA, which measured faster.
// Shared memory: twiddle area | sigma rows[2][N] | sbuf[2 SP_ROW].
template <typename T, int LOGN, bool BATCH, bool TC>
__global__ void __launch_bounds__(KShape<LOGN>::ROW_THREADS) k_row_fwd_m(SolveArgs<T> a0, BatchView<T> bv)
{
    const int2 wm = BATCH ? bv.map[blockIdx.y] : make_int2(0, 0);
    const SolveArgs<T> &a = BATCH ? bv.args[wm.x] : a0;
    using C = typename Cx<T>::C;
    using C2 = typename Cx<T>::C2;
    using K = KShape<LOGN>;
    constexpr int N = K::N, Q = K::Q, SP = K::SP_ROW;
    extern __shared__ __align__(16) unsigned char smem_tc[];
    constexpr int TCT = tc_tiles(KShape<LOGN>::ROW_THREADS, 1);
    constexpr int TCR = tc_round(LOGN, TCT, KK_ROW_FWD_M);
    static_assert(!TC || sizeof(T) == 4, "tensor-core tiles take FP32 data");
    unsigned char *smem_raw = smem_tc + (TC ? tc_smem_bytes(TCR) : 0);
    TcCtx tcx;
    if constexpr (TC)
        tc_begin(tcx, smem_tc, TCT, TCR, a.status, a.wait_cycles, a.inject);
    C *tw = reinterpret_cast<C *>(smem_raw);
    T *srow = reinterpret_cast<T *>(smem_raw + tw_bytes<C>(a.tw_entries));
    C *sbuf = reinterpret_cast<C *>(srow + 2 * N);
    __shared__ int rim_bad;
    const int t = threadIdx.x;
    if (t == 0)
        rim_bad = 0;
    cp_block(tw, a.tw, tw_bytes<C>(a.tw_entries));
    cp_block(srow, a.src[0] + (size_t)(2 * blockIdx.x) * N, 2 * (size_t)N * sizeof(T));
    cp_commit();
    const bool active = t < 2 * Q;
    const int b = active ? t / Q : 0, j = active ? t - b * Q : 0;
    const TwLayout tl = tw_layout(F16<LOGN>::twlen, N);
    constexpr bool WALK = TC && !BATCH;  // the other instances take one row pair per CTA
    for (int rp = blockIdx.x; rp < N / 2; rp += WALK ? (int)gridDim.x : N / 2) {
        const int r0 = 2 * rp;
        cp_wait<0>();
        __syncthreads();  // rows r0, r0 + 1 staged; the previous pair's bins have been read
        {
            bool bad = false;
            const int nl = a.n_log;  // the patch's own cells (zero beyond them in an embedded array)
            if (r0 == 0 || r0 == nl - 2) {
                for (int i = t; i < 2 * N; i += K::ROW_THREADS)
                    bad |= srow[i] != T(0);
            } else if (t < 8 && r0 < nl) {
                const int col = (t & 3) < 2 ? (t & 3) : nl - 4 + (t & 3);  // 0, 1, n-2, n-1
                bad = srow[(t >> 2) * N + col] != T(0);
            }
            if (bad)
                rim_bad = 1;
        }
        C v[1][16];
        if (active) {
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int c = j + u * Q;
                C z = hmk<C>(srow[c], srow[N + c]);
                if (b)
                    z = hmul(z, twist(tw, tl, j, u));
                v[0][u] = z;
            }
        }
        if (WALK && rp + (int)gridDim.x < N / 2) {  // uniform over the block
            __syncthreads();  // every thread has read the rows
            cp_block(srow, a.src[0] + (size_t)(2 * (rp + gridDim.x)) * N, 2 * (size_t)N * sizeof(T));
            cp_commit();
        }
        constexpr int HB = TC ? 0 : K::HB_ROW;
        fft_ct<C, false, LOGN, 1, TC, HB>(v, sbuf + b * SP, SP, j, active, tw, &tcx, b);
        __syncthreads();
        if (active) {
#pragma unroll
            for (int u = 0; u < 16; ++u)
                sbuf[b * SP + pad16(j + u * Q)] = v[0][u];
        }
        __syncthreads();
        C2 *out = reinterpret_cast<C2 *>(a.fwd);
        for (int kx = t; kx <= N; kx += K::ROW_THREADS) {
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
    cp_wait<0>();
    __syncthreads();
    if (t == 0 && rim_bad)
        atomicOr(a.status, STATUS_RIM_NONZERO);
    if constexpr (TC)
        tc_end(tcx, TCT);
}

// k_row_fwd_m (FP32, no tensor-core tiles, no batch view) with two row pairs
// per CTA: group g = t / (N/8) of 2 N/16 threads transforms row pair
// 2 blockIdx.x + g exactly as k_row_fwd_m transforms its one (parity halves on
// named barriers 1 + 2 g + half), and in the store phase two neighbouring
// lanes write the two row pairs of one bin, rows 4 blockIdx.x .. + 3: 32
// contiguous bytes, one whole sector, where a CTA of one row pair writes 16.
// Shared memory: twiddle area | sigma rows [4][N] | sbuf [2 pairs][2 halves][SP_ROW].
template <int LOGN>
__global__ void __launch_bounds__((1 << LOGN) / 4) k_row_fwd_m2(SolveArgs<float> a)
{
    using C = float2;
    using C2 = float4;
    using K = KShape<LOGN>;
    constexpr int N = K::N, Q = K::Q, SP = K::SP_ROW, T2 = 2 * Q;
    static_assert(Q >= 32, "whole warps per parity half");
    extern __shared__ __align__(16) unsigned char smem_f2[];
    C *tw = reinterpret_cast<C *>(smem_f2);
    float *srow = reinterpret_cast<float *>(smem_f2 + tw_bytes<C>(a.tw_entries));
    C *sbuf = reinterpret_cast<C *>(srow + 4 * N);
    __shared__ int rim_bad;
    const int t = threadIdx.x;
    const int g = t / T2, tg = t - g * T2, b = tg / Q, j = tg - b * Q;
    if (t == 0)
        rim_bad = 0;
    cp_block(tw, a.tw, tw_bytes<C>(a.tw_entries));
    cp_block(srow, a.src[0] + (size_t)(4 * blockIdx.x) * N, 4 * (size_t)N * sizeof(float));  // both pairs' rows
    cp_commit();
    cp_wait<0>();
    __syncthreads();
    const int r0 = 4 * (int)blockIdx.x + 2 * g;
    const float *rows = srow + 2 * g * N;
    {
        bool bad = false;
        const int nl = a.n_log;  // the patch's own cells (zero beyond them in an embedded array)
        if (r0 == 0 || r0 == nl - 2) {
            for (int i = tg; i < 2 * N; i += T2)
                bad |= rows[i] != 0.0f;
        } else if (tg < 8 && r0 < nl) {
            const int col = (tg & 3) < 2 ? (tg & 3) : nl - 4 + (tg & 3);  // 0, 1, n-2, n-1
            bad = rows[(tg >> 2) * N + col] != 0.0f;
        }
        if (bad)
            rim_bad = 1;
    }
    const TwLayout tl = tw_layout(F16<LOGN>::twlen, N);
    C v[1][16];
#pragma unroll
    for (int u = 0; u < 16; ++u) {
        const int c = j + u * Q;
        C z = hmk<C>(rows[c], rows[N + c]);
        if (b)
            z = hmul(z, twist(tw, tl, j, u));
        v[0][u] = z;
    }
    fft_ct<C, false, LOGN, 1, false, Q>(v, sbuf + (2 * g + b) * SP, SP, j, true, tw, nullptr, 2 * g + b);
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 16; ++u)
        sbuf[(2 * g + b) * SP + pad16(j + u * Q)] = v[0][u];
    __syncthreads();
    C2 *out = reinterpret_cast<C2 *>(a.fwd);
    for (int e = t; e < 2 * (N + 1); e += 4 * Q) {  // e = 2 kx + pair: neighbouring lanes, one sector
        const int pr = e & 1, kx = e >> 1;
        const int bb = kx & 1, k = kx >> 1;
        const int km = (N - bb - k) & (N - 1);
        const C Z = sbuf[(2 * pr + bb) * SP + pad16(k)];
        const C Zm = sbuf[(2 * pr + bb) * SP + pad16(km)];
        C2 o;
        o.x = 0.5f * (Z.x + Zm.x);
        o.y = 0.5f * (Z.y - Zm.y);
        o.z = 0.5f * (Z.y + Zm.y);
        o.w = -0.5f * (Z.x - Zm.x);
        out[((size_t)kx * N + 4 * blockIdx.x + 2 * pr) >> 1] = o;
    }
    if (t == 0 && rim_bad)
        atomicOr(a.status, STATUS_RIM_NONZERO);
}

// k_row_fwd_m2 with the structure of k_row_inv2x: one thread per slot j
// carries both parity halves of a row pair's transform (x and x W_P^n as two
// sequences) with the slot's stage twiddles in registers, and the CTA walks
// its items of two row pairs (rows 4q .. 4q + 3): the item's four sigma rows
// are staged by cp.async, the pairs are transformed one after the other, the
// first pair's bins wait in their own buffer while the second is transformed,
// and the next item's rows are copied in as soon as the second pair is in
// registers.  Neighbouring lanes then store the two pairs' values of one bin,
// one 32-byte sector.  G = 256 / (N/16) groups of N/16 threads per CTA, each
// walking its own items on its own named barrier.  Also verifies the zero rim
// as k_row_fwd_m does.  FP32, N >= 1024, one patch, no batch view.
// Shared memory per group: sigma rows [4][N] | exchange buffers [2][SP_ROW] |
// 32 bytes | first pair's bins [2][SP_ROW].  (The 32 bytes put the two pairs'
// bins of one index in different banks: the unpack of a quarter warp reads
// four bins of each half of each pair.)
template <int LOGN>
struct KFx {
    static constexpr int N = 1 << LOGN, Q = N >> 4;
    static constexpr int G = Q >= 256 ? 1 : 256 / Q;
    static constexpr int THREADS = G * Q;
    static constexpr size_t XB = 2 * (size_t)KShape<LOGN>::SP_ROW * 8;
    static constexpr size_t GROUP_BYTES = 4 * (size_t)N * 4 + 2 * XB + 32;
    static constexpr size_t SMEM = G * GROUP_BYTES;
};

template <int LOGN, int PLAN>
__global__ void __launch_bounds__(KFx<LOGN>::THREADS, 1) k_row_fwd_x(const __grid_constant__ SolveArgs<float> a)
{
    using C = float2;
    using C2 = float4;
    using R = KFx<LOGN>;
    using P = FR<LOGN, PLAN>;
    constexpr int N = R::N, Q = R::Q, SP = KShape<LOGN>::SP_ROW;
    static_assert(Q >= 64, "named group barriers need whole warps");
    extern __shared__ __align__(16) unsigned char smem_fx[];
    const int t = threadIdx.x;
    const int g = t / Q, j = t - g * Q;
    unsigned char *gb = smem_fx + (size_t)g * R::GROUP_BYTES;
    float *rows = reinterpret_cast<float *>(gb);
    C *xb = reinterpret_cast<C *>(gb + 4 * (size_t)N * 4);
    C *za = xb + 2 * SP + 4;
    __shared__ int rim_bad;
    if (t == 0)
        rim_bad = 0;
    __syncthreads();
    const unsigned bar = 1 + g;
    const int nl = a.n_log;
    const int items = N / 4;
    C trw[P::NST - 1][15];
    load_twiddles_rt<C, LOGN, PLAN>(trw, a.twn, j);
    const TwLayout tl = tw_layout(F16<LOGN>::twlen, N);
    const C wj = a.tw[tl.base + j];  // W_P^j
    auto twist_u = [&](int u) { return hmul(wj, hmk<C>((float)kW32c[u], (float)-kW32s[u])); };
    const float *src = a.src[0];
    auto stage = [&](int it) {  // this group's threads: rows 4 it .. 4 it + 3 (contiguous)
        const char *s = reinterpret_cast<const char *>(src + (size_t)(4 * it) * N);
        for (int o = j * 16; o < 4 * N * 4; o += Q * 16)
            cp16(reinterpret_cast<char *>(rows) + o, s + o);
        cp_commit();
    };
    const int step = (int)gridDim.x * R::G;
    int it = (int)blockIdx.x * R::G + g;
    if (it < items)
        stage(it);
    bool bad = false;
    for (; it < items; it += step) {  // uniform over the group
        cp_wait<0>();
        group_sync(bar, Q);  // the item's rows are staged; the previous item's bins are stored
#pragma unroll
        for (int h = 0; h < 2; ++h) {  // the zero rim: rows 0, 1 and nl-2, nl-1 whole, columns 0, 1, nl-2, nl-1
            const int r0 = 4 * it + 2 * h;
            const float *rp = rows + 2 * h * N;
            if (r0 == 0 || r0 == nl - 2) {
                for (int i = j; i < 2 * N; i += Q)
                    bad |= rp[i] != 0.0f;
            } else if (j < 8 && r0 < nl) {
                const int col = (j & 3) < 2 ? (j & 3) : nl - 4 + (j & 3);
                bad |= rp[(j >> 2) * N + col] != 0.0f;
            }
        }
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
            C v[2][16];
            const float *rp = rows + 2 * h * N;
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int c = j + u * Q;
                const C z = hmk<C>(rp[c], rp[N + c]);
                v[0][u] = z;
                v[1][u] = hmul(z, twist_u(u));
            }
            if (h == 1) {
                group_sync(bar, Q);  // every thread has read the rows
                if (it + step < items)
                    stage(it + step);
            }
            fft_stages_rt<C, false, LOGN, PLAN, 2, 0>(v, xb, SP, j, trw, bar, Q);
            group_sync(bar, Q);  // the last stage's reads of the exchange buffers are done
            C *zb = h ? xb : za;
#pragma unroll
            for (int b = 0; b < 2; ++b)
#pragma unroll
                for (int u = 0; u < 16; ++u)
                    zb[b * SP + pad16(j + u * Q)] = v[b][u];
        }
        group_sync(bar, Q);  // both pairs' bins are in shared memory
        // X_a = (Z + conj Z~)/2, X_b = (Z - conj Z~)/(2i); Z~ = bin -kx, same parity half
        C2 *out = reinterpret_cast<C2 *>(a.fwd);
        for (int e = j; e < 2 * (N + 1); e += Q) {  // e = 2 kx + pair: neighbouring lanes, one sector
            const int pr = e & 1, kx = e >> 1;
            const C *zb = pr ? xb : za;
            const int bb = kx & 1, k = kx >> 1;
            const int km = (N - bb - k) & (N - 1);
            const C Z = zb[bb * SP + pad16(k)];
            const C Zm = zb[bb * SP + pad16(km)];
            C2 o;
            o.x = 0.5f * (Z.x + Zm.x);
            o.y = 0.5f * (Z.y - Zm.y);
            o.z = 0.5f * (Z.y + Zm.y);
            o.w = -0.5f * (Z.x - Zm.x);
            out[((size_t)kx * N + 4 * it + 2 * pr) >> 1] = o;
        }
    }
    cp_wait<0>();  // nothing in flight at exit
    if (bad)
        rim_bad = 1;
    __syncthreads();
    if (t == 0 && rim_bad)
        atomicOr(a.status, STATUS_RIM_NONZERO);
}

// The three-field forward row pass (k_row_fwd) of a plan of one patch without
// the zero rim, on the register-twiddle engine: one thread per slot j carries
// both parity halves of a row pair's transform with the slot's stage twiddles
// in registers, and the CTA walks the row pairs.  A row pair's fields (sigma,
// its x slope, its y slope, exactly as k_row_fwd forms them) all come from the
// four sigma rows r0 - 1 .. r0 + 2 (clamped to the array), staged once by
// cp.async into one of two buffers: the next pair's rows are copied in while
// this pair's three fields are transformed one after the other.  The bins of a
// field are unpacked through the exchange buffers and stored in 16-byte pieces
// (one row pair).  G = 256 / (N/16) groups of N/16 threads per CTA, each
// walking its own pairs on its own named barrier.  FP32, N >= 1024, no batch
// view.  Shared memory per group: sigma rows [2][4][N] | exchange buffers
// [2][SP_ROW].
template <int LOGN>
struct KF3x {
    static constexpr int N = 1 << LOGN, Q = N >> 4;
    static constexpr int G = Q >= 256 ? 1 : 256 / Q;
    static constexpr int THREADS = G * Q;
    static constexpr size_t ROWS = 4 * (size_t)N * 4;
    static constexpr size_t GROUP_BYTES = 2 * ROWS + 2 * (size_t)KShape<LOGN>::SP_ROW * 8;
    static constexpr size_t SMEM = G * GROUP_BYTES;
};

template <int LOGN, int PLAN>
__global__ void __launch_bounds__(KF3x<LOGN>::THREADS, 1) k_row_fwd3x(const __grid_constant__ SolveArgs<float> a)
{
    using C = float2;
    using C2 = float4;
    using R = KF3x<LOGN>;
    using P = FR<LOGN, PLAN>;
    constexpr int N = R::N, Q = R::Q, SP = KShape<LOGN>::SP_ROW;
    static_assert(Q >= 64, "named group barriers need whole warps");
    extern __shared__ __align__(16) unsigned char smem_f3x[];
    const int t = threadIdx.x;
    const int g = t / Q, j = t - g * Q;
    unsigned char *gb = smem_f3x + (size_t)g * R::GROUP_BYTES;
    C *xb = reinterpret_cast<C *>(gb + 2 * R::ROWS);
    const unsigned bar = 1 + g;
    const int nl = a.n_log;
    const FwdSlab sl = a.slabs[0];
    const int items = N / 2;
    C trw[P::NST - 1][15];
    load_twiddles_rt<C, LOGN, PLAN>(trw, a.twn, j);
    const TwLayout tl = tw_layout(F16<LOGN>::twlen, N);
    const C wj = a.tw[tl.base + j];  // W_P^j
    auto twist_u = [&](int u) { return hmul(wj, hmk<C>((float)kW32c[u], (float)-kW32s[u])); };
    const float *src = a.src[0];
    auto first_row = [&](int it) { return min(max(2 * it - 1, 0), N - 4); };
    auto stage = [&](int it, int buf) {  // this group's threads: rows first_row .. + 3 (contiguous)
        const char *s = reinterpret_cast<const char *>(src + (size_t)first_row(it) * N);
        char *d = reinterpret_cast<char *>(gb + (size_t)buf * R::ROWS);
        for (int o = j * 16; o < 4 * N * 4; o += Q * 16)
            cp16(d + o, s + o);
        cp_commit();
    };
    const int step = (int)gridDim.x * R::G;
    int it = (int)blockIdx.x * R::G + g;
    if (it < items)
        stage(it, 0);
    C2 *out = reinterpret_cast<C2 *>(a.fwd + sl.off);
    for (int buf = 0; it < items; it += step, buf ^= 1) {  // uniform over the group
        cp_wait<0>();
        group_sync(bar, Q);  // this pair's rows are staged; the other buffer is free
        if (it + step < items)
            stage(it + step, buf ^ 1);
        const int r0 = 2 * it, s0 = first_row(it);
        const float *rows = reinterpret_cast<const float *>(gb + (size_t)buf * R::ROWS);
        auto row = [&](int jj) { return rows + (size_t)(jj - s0) * N; };
        auto field = [&](auto fcv) {  // one field after the other, each compiled on its own
            constexpr int f = decltype(fcv)::value;
            C v[2][16];
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int i = j + u * Q;
                float fv[2] = {0.0f, 0.0f};
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int jj = r0 + h;
                    if (i >= nl || jj >= nl)
                        continue;
                    if constexpr (f == 0) {
                        fv[h] = row(jj)[i];
                    } else if constexpr (f == 1) {
                        const float *r = row(jj);
                        const int il = i == 0 ? 0 : i - 1, ir = i == nl - 1 ? nl - 1 : i + 1;
                        const float d = r[ir] - r[il];
                        fv[h] = (ir - il == 2) ? 0.5f * d : d;
                    } else {
                        const int jd = max(jj - 1, 0), ju = min(jj + 1, nl - 1);
                        const float d = row(min(ju, N - 1))[i] - row(min(jd, N - 1))[i];
                        fv[h] = (jj == 0 || jj == nl - 1) ? d : 0.5f * d;
                    }
                }
                const C z = hmk<C>(fv[0], fv[1]);
                v[0][u] = z;
                v[1][u] = hmul(z, twist_u(u));
            }
            fft_stages_rt<C, false, LOGN, PLAN, 2, 0>(v, xb, SP, j, trw, bar, Q);
            group_sync(bar, Q);  // the last stage's reads of the exchange buffers are done
#pragma unroll
            for (int b = 0; b < 2; ++b)
#pragma unroll
                for (int u = 0; u < 16; ++u)
                    xb[b * SP + pad16(j + u * Q)] = v[b][u];
            group_sync(bar, Q);
            // X_a = (Z + conj Z~)/2, X_b = (Z - conj Z~)/(2i); Z~ = bin -kx, same parity half
            for (int kx = j; kx <= N; kx += Q) {
                const int bb = kx & 1, k = kx >> 1;
                const int km = (N - bb - k) & (N - 1);
                const C Z = xb[bb * SP + pad16(k)];
                const C Zm = xb[bb * SP + pad16(km)];
                C2 o;
                o.x = 0.5f * (Z.x + Zm.x);
                o.y = 0.5f * (Z.y - Zm.y);
                o.z = 0.5f * (Z.y + Zm.y);
                o.w = -0.5f * (Z.x - Zm.x);
                out[(((size_t)f * (N + 1) + kx) * sl.rows + r0) >> 1] = o;
            }
            // the next field's transform writes the exchange buffers only after
            // its first stage's barrier, when every thread has read them here
        };
        field(std::integral_constant<int, 0>{});
        field(std::integral_constant<int, 1>{});
        field(std::integral_constant<int, 2>{});
    }
    cp_wait<0>();  // nothing in flight at exit
}

// Column pass of a SGF_PLAN_ZERO_RIM plan: one forward transform, the two
// merged spectra (Fx^ = Gx^ sigma^, Fy^ = Gy^ sigma^, both imaginary), and the
// two inverse transforms one after the other; parity halves folded through
// distributed shared memory.  The column and the spectrum half rows are read
// straight into registers (coalesced), Fy^ waits in shared memory while Fx^ is
// transformed, so a thread holds one sequence at a time and three CTAs fit on
// an SM.  The tensor-core instance is launched with the clusters that fit at
// once, each walking the columns.  Shared memory: twiddle area | sbuf[SPC]
// (exchanges, then the fold) | park[N] (Fy^ in slot order).
template <typename T, int LOGN, bool BATCH, bool TC>
__global__ void __cluster_dims__(2, 1, 1)
    __launch_bounds__(KShape<LOGN>::COL_THREADS, sizeof(T) == 4 && !TC ? 3 : 1) k_col_m(SolveArgs<T> a0, BatchView<T> bv)
{
    const int2 wm = BATCH ? bv.map[blockIdx.y] : make_int2(0, 0);
    const SolveArgs<T> &a = BATCH ? bv.args[wm.x] : a0;
    using C = typename Cx<T>::C;
    using K = KShape<LOGN>;
    constexpr int N = K::N, Q = K::Q, QS = quarter_stride(N), HQ = quarter_half(N);
    constexpr int SPC = col_sp<C>(N);
    extern __shared__ __align__(16) unsigned char smem_tc[];
    constexpr int TCT = tc_tiles(KShape<LOGN>::COL_THREADS, 1);
    constexpr int TCR = tc_round(LOGN, TCT, KK_COL_M);
    static_assert(!TC || sizeof(T) == 4, "tensor-core tiles take FP32 data");
    unsigned char *smem_raw = smem_tc + (TC ? tc_smem_bytes(TCR) : 0);
    TcCtx tcx;
    if constexpr (TC)
        tc_begin(tcx, smem_tc, TCT, TCR, a.status, a.wait_cycles, a.inject);
    C *tw = reinterpret_cast<C *>(smem_raw);
    C *sbuf = reinterpret_cast<C *>(smem_raw + tw_bytes<C>(a.tw_entries));
    C *park = sbuf + SPC;
    cg::cluster_group cluster = cg::this_cluster();
    const int b = (int)cluster.block_rank();
    const int t = threadIdx.x;
    const bool active = t < Q;
    const int j = active ? t : 0;
    const TwLayout tl = tw_layout(F16<LOGN>::twlen, N);
    cp_block(tw, a.tw, tw_bytes<C>(a.tw_entries));
    cp_commit();
    // tensor-core instances: the resident clusters walk the columns (tiles and tensor memory set up once)
    constexpr bool WALK = TC && !BATCH;
    for (int kx = blockIdx.x >> 1; kx <= N; kx += WALK ? (int)(gridDim.x >> 1) : N + 1) {
        const T *gxr = reinterpret_cast<const T *>(a.spec) + (size_t)kx * QS + b * HQ;
        const T *gyr = reinterpret_cast<const T *>(a.spec) + ((size_t)(N + 1) + kx) * QS + b * HQ;
        C v[1][16];
        if (active) {
            const C *col = a.fwd + (size_t)kx * N;
#pragma unroll
            for (int u = 0; u < 16; ++u)
                v[0][u] = col[j + u * Q];
        }
        cp_wait<0>();
        __syncthreads();
        if (active && b) {
#pragma unroll
            for (int u = 0; u < 16; ++u)
                v[0][u] = hmul(v[0][u], twist(tw, tl, j, u));
        }
        fft_ct<C, false, LOGN, 1, TC>(v, sbuf, SPC, j, active, tw, &tcx);
        if (active) {
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int kp = j + u * Q;
                const bool hi = 2 * kp + b > N;
                const int q = hi ? N - kp - b : kp;
                const T gx = __ldg(gxr + q);                               // Gx even in ky
                const T gy = hi ? -__ldg(gyr + q) : __ldg(gyr + q);        // Gy odd in ky
                park[u * Q + j] = hmk<C>(-gy * v[0][u].y, gy * v[0][u].x);  // i gy v
                v[0][u] = hmk<C>(-gx * v[0][u].y, gx * v[0][u].x);          // i gx v
            }
        }
        C *const out = a.bwd;
#pragma unroll 1
        for (int comp = 0; comp < 2; ++comp) {
            if (comp == 1 && active) {
#pragma unroll
                for (int u = 0; u < 16; ++u)
                    v[0][u] = park[u * Q + j];
            }
            // y[n] = even[n] + W_P^{-n} odd[n]
            fft_ct<C, true, LOGN, 1, TC>(v, sbuf, SPC, j, active, tw, &tcx);
            cluster.sync();  // both CTAs are done with their exchange buffers
            if (b == 1 && active) {
                C *dst = cluster.map_shared_rank(sbuf, 0);
#pragma unroll
                for (int u = 0; u < 16; ++u)
                    dst[j + u * Q] = hmulc(v[0][u], twist(tw, tl, j, u));
            }
            cluster.sync();
            if (b == 0 && active) {
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    const int n = j + u * Q;
                    out[bwd_index(N, N, comp, kx, n)] = hadd(v[0][u], sbuf[n]);
                }
            }
        }
    }
    if constexpr (TC)
        tc_end(tcx, TCT);
}

// The same column pass with both inverse transforms in flight at once (B = 2
// sequences per thread share the barriers): fewer barriers, twice the
// registers, two CTAs per SM.  The column and the spectrum half rows are
// staged with asynchronous copies.  The tensor-core instance is launched with
// the clusters that fit at once, each walking the columns.  Shared memory:
// twiddle area | sbuf[SPC] | column[N] | Gx, Gy half rows; the second
// sequence and the 2N fold reuse sbuf + column.
template <typename T, int LOGN, bool BATCH, bool TC>
__global__ void __cluster_dims__(2, 1, 1)
    __launch_bounds__(KShape<LOGN>::COL_THREADS, sizeof(T) == 4 && !TC ? 2 : 1) k_col_md(SolveArgs<T> a0, BatchView<T> bv)
{
    const int2 wm = BATCH ? bv.map[blockIdx.y] : make_int2(0, 0);
    const SolveArgs<T> &a = BATCH ? bv.args[wm.x] : a0;
    using C = typename Cx<T>::C;
    using K = KShape<LOGN>;
    constexpr int N = K::N, Q = K::Q, QS = quarter_stride(N), HQ = quarter_half(N);
    constexpr int SPC = col_sp<C>(N);
    extern __shared__ __align__(16) unsigned char smem_tc[];
    constexpr int TCT = tc_tiles(KShape<LOGN>::COL_THREADS, 2);
    constexpr int TCR = tc_round(LOGN, TCT, KK_COL_MD);
    static_assert(!TC || sizeof(T) == 4, "tensor-core tiles take FP32 data");
    unsigned char *smem_raw = smem_tc + (TC ? tc_smem_bytes(TCR) : 0);
    TcCtx tcx;
    if constexpr (TC)
        tc_begin(tcx, smem_tc, TCT, TCR, a.status, a.wait_cycles, a.inject);
    C *tw = reinterpret_cast<C *>(smem_raw);
    C *sbuf = reinterpret_cast<C *>(smem_raw + tw_bytes<C>(a.tw_entries));
    C *col = sbuf + SPC;
    T *gsp = reinterpret_cast<T *>(col + N);
    cg::cluster_group cluster = cg::this_cluster();
    const int b = (int)cluster.block_rank();
    const int t = threadIdx.x;
    const bool active = t < Q;
    const int j = active ? t : 0;
    const TwLayout tl = tw_layout(F16<LOGN>::twlen, N);
    const T *spec = reinterpret_cast<const T *>(a.spec);
    cp_block(tw, a.tw, tw_bytes<C>(a.tw_entries));
    // tensor-core instances: the resident clusters walk the columns (tiles and tensor memory set up once)
    constexpr bool WALK = TC && !BATCH;
    for (int kx = blockIdx.x >> 1; kx <= N; kx += WALK ? (int)(gridDim.x >> 1) : N + 1) {
        if (WALK && kx != (int)(blockIdx.x >> 1))
            __syncthreads();  // the previous column's fold (over sbuf and the column) has been read
        cp_block(col, a.fwd + (size_t)kx * N, (size_t)N * sizeof(C));
        cp_block(gsp, spec + (size_t)kx * QS + b * HQ, (size_t)HQ * sizeof(T));
        cp_block(gsp + HQ, spec + ((size_t)(N + 1) + kx) * QS + b * HQ, (size_t)HQ * sizeof(T));
        cp_commit();
        cp_wait<0>();
        __syncthreads();
        C acc[2][16];
        {
            C v[1][16];
            if (active) {
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    C x = col[j + u * Q];
                    if (b)
                        x = hmul(x, twist(tw, tl, j, u));
                    v[0][u] = x;
                }
            }
            fft_ct<C, false, LOGN, 1, TC>(v, sbuf, SPC, j, active, tw, &tcx);
            if (active) {
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    const int kp = j + u * Q;
                    const bool hi = 2 * kp + b > N;
                    const int q = hi ? N - kp - b : kp;
                    const T gx = gsp[q];                           // Gx even in ky
                    const T gy = hi ? -gsp[HQ + q] : gsp[HQ + q];  // Gy odd in ky
                    acc[0][u] = hmk<C>(-gx * v[0][u].y, gx * v[0][u].x);  // i gx v
                    acc[1][u] = hmk<C>(-gy * v[0][u].y, gy * v[0][u].x);
                }
            }
        }
        fft_ct<C, true, LOGN, 2, TC>(acc, sbuf, SPC, j, active, tw, &tcx);  // second sequence over the column
        C *fold = sbuf;
        cluster.sync();
        if (b == 1 && active) {
            C *dst = cluster.map_shared_rank(fold, 0);
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int n = j + u * Q;
                const C w = twist(tw, tl, j, u);
                dst[n] = hmulc(acc[0][u], w);
                dst[N + n] = hmulc(acc[1][u], w);
            }
        }
        cluster.sync();
        if (b == 0 && active) {
            C *dst = a.bwd;
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int n = j + u * Q;
                dst[bwd_index(N, N, 0, kx, n)] = hadd(acc[0][u], fold[n]);
                dst[bwd_index(N, N, 1, kx, n)] = hadd(acc[1][u], fold[N + n]);
            }
        }
    }
    if constexpr (TC)
        tc_end(tcx, TCT);
}

// The zero-rim column pass with one CTA per column holding both parity halves
// (thread t: half t / (N/16), slot t mod (N/16)): the column is staged once and
// the odd half is folded through shared memory under the CTA barrier, with no
// cluster.  Both inverse transforms in flight (two sequences per thread).
// The CTA walks the columns kx = blockIdx.x, blockIdx.x + gridDim.x, ... (one
// resident CTA per SM holds the whole shared memory, so consecutive columns of
// separate CTAs could not overlap): once the forward transform and the
// spectral product have consumed a column's staging, the next column's input
// is copied in behind the inverse transforms.  Batches launch one CTA per
// (column, work item) and walk one column.
// Shared memory: twiddle area | column[N] | Gx, Gy half rows of both halves |
// exchange buffers, half b's two sequences at sbuf + 2 b SPC (then the fold).
// NC = 2: the forces (Gx, Gy); NC = 1: the potential (Gphi alone, one inverse transform).
template <typename T, int LOGN, bool BATCH, bool TC, int NC = 2>
__global__ void __launch_bounds__(KShape<LOGN>::ROW_THREADS, 1) k_col_mw(SolveArgs<T> a0, BatchView<T> bv)
{
    const int2 wm = BATCH ? bv.map[blockIdx.y] : make_int2(0, 0);
    const SolveArgs<T> &a = BATCH ? bv.args[wm.x] : a0;
    using C = typename Cx<T>::C;
    using K = KShape<LOGN>;
    constexpr int N = K::N, Q = K::Q, QS = quarter_stride(N), HQ = quarter_half(N);
    constexpr int SPC = col_sp<C>(N);
    extern __shared__ __align__(16) unsigned char smem_tc[];
    constexpr int TCT = tc_tiles(KShape<LOGN>::ROW_THREADS, 2);
    constexpr int TCR = tc_round(LOGN, TCT, KK_COL_MW);
    static_assert(!TC || sizeof(T) == 4, "tensor-core tiles take FP32 data");
    unsigned char *smem_raw = smem_tc + (TC ? tc_smem_bytes(TCR) : 0);
    TcCtx tcx;
    if constexpr (TC)
        tc_begin(tcx, smem_tc, TCT, TCR, a.status, a.wait_cycles, a.inject);
    C *tw = reinterpret_cast<C *>(smem_raw);
    C *col = reinterpret_cast<C *>(smem_raw + tw_bytes<C>(a.tw_entries));
    T *gsp = reinterpret_cast<T *>(col + N);  // [half][Gx, Gy][HQ]
    C *sbuf = reinterpret_cast<C *>(gsp + 4 * HQ);
    const int t = threadIdx.x;
    const bool active = t < 2 * Q;
    const int b = active ? t / Q : 0, j = active ? t - b * Q : 0;
    const TwLayout tl = tw_layout(F16<LOGN>::twlen, N);
    const T *spec = reinterpret_cast<const T *>(a.spec);
    constexpr bool two = NC == 2;  // the forces (Gx, Gy); else the potential (Gphi alone)
    auto stage = [&](int kx) {  // whole block: column kx of the forward slab and its spectra half rows
        cp_block(col, a.fwd + (size_t)kx * N, (size_t)N * sizeof(C));
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            cp_block(gsp + (2 * h) * HQ, spec + (size_t)kx * QS + h * HQ, (size_t)HQ * sizeof(T));
            if (two)
                cp_block(gsp + (2 * h + 1) * HQ, spec + ((size_t)(N + 1) + kx) * QS + h * HQ, (size_t)HQ * sizeof(T));
        }
        cp_commit();
    };
    cp_block(tw, a.tw, tw_bytes<C>(a.tw_entries));
    stage(blockIdx.x);
    for (int kx = blockIdx.x; kx <= N; kx += gridDim.x) {
        cp_wait<0>();
        __syncthreads();  // column kx staged; the previous column's fold has been read
        C acc[2][16];
        {
            C v[1][16];
            if (active) {
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    C x = col[j + u * Q];
                    if (b)
                        x = hmul(x, twist(tw, tl, j, u));
                    v[0][u] = x;
                }
            }
            // each half transforms in its own buffers until the fold: half barriers
            fft_ct<C, false, LOGN, 1, TC, TC ? 0 : K::HB_ROW>(v, sbuf + 2 * b * SPC, SPC, j, active, tw, &tcx, b);
            if constexpr (two) {
                if (active) {
                    const T *gx_r = gsp + (2 * b) * HQ, *gy_r = gsp + (2 * b + 1) * HQ;
#pragma unroll
                    for (int u = 0; u < 16; ++u) {
                        const int kp = j + u * Q;
                        const bool hi = 2 * kp + b > N;
                        const int q = hi ? N - kp - b : kp;
                        const T gx = gx_r[q];                        // Gx even in ky
                        const T gy = hi ? -gy_r[q] : gy_r[q];        // Gy odd in ky
                        acc[0][u] = hmk<C>(-gx * v[0][u].y, gx * v[0][u].x);  // i gx v
                        acc[1][u] = hmk<C>(-gy * v[0][u].y, gy * v[0][u].x);
                    }
                }
            } else if (active) {
                const T *gp_r = gsp + (2 * b) * HQ;
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    const int kp = j + u * Q;
                    const int q = 2 * kp + b > N ? N - kp - b : kp;
                    const T gp = gp_r[q];  // Gphi real, even in ky
                    acc[0][u] = hmk<C>(gp * v[0][u].x, gp * v[0][u].y);
                }
            }
        }
        if (kx + (int)gridDim.x <= N) {  // uniform over the block
            __syncthreads();  // every thread is done with the column and the spectra rows
            stage(kx + gridDim.x);
        }
        C *dst = a.bwd;
        if constexpr (!two) {  // the potential: one inverse transform, the stores split by n between the halves
            fft_ct<C, true, LOGN, 1, TC, TC ? 0 : K::HB_ROW>(acc, sbuf + 2 * b * SPC, SPC, j, active, tw, &tcx, b);
            __syncthreads();  // every exchange buffer has been read
            C *fold = sbuf;
            if (active) {
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    const int n = j + u * Q;
                    if (b == 1 && u < 8)
                        fold[n] = hmulc(acc[0][u], twist(tw, tl, j, u));
                    else if (b == 0 && u >= 8)
                        fold[n] = acc[0][u];
                }
            }
            __syncthreads();
            if (active) {
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    const int n = j + u * Q;
                    if (b == 0 && u < 8)
                        dst[bwd_index(N, N, 0, kx, n)] = hadd(acc[0][u], fold[n]);
                    else if (b == 1 && u >= 8)
                        dst[bwd_index(N, N, 0, kx, n)] = hadd(fold[n], hmulc(acc[0][u], twist(tw, tl, j, u)));
                }
            }
        } else {
            fft_ct<C, true, LOGN, 2, TC, TC ? 0 : K::HB_ROW>(acc, sbuf + 2 * b * SPC, SPC, j, active, tw, &tcx, b);
            __syncthreads();  // every exchange buffer has been read
            // fold y = even + W_P^{-n} odd, one component per half: the odd half hands over
            // Fx's twisted values, the even half Fy's own, and each stores one component
            C *fold = sbuf;
            if (active) {
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    const int n = j + u * Q;
                    if (b == 1)
                        fold[n] = hmulc(acc[0][u], twist(tw, tl, j, u));
                    else
                        fold[N + n] = acc[1][u];
                }
            }
            __syncthreads();
            if (active) {
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    const int n = j + u * Q;
                    if (b == 0)
                        dst[bwd_index(N, N, 0, kx, n)] = hadd(acc[0][u], fold[n]);
                    else
                        dst[bwd_index(N, N, 1, kx, n)] = hadd(fold[N + n], hmulc(acc[1][u], twist(tw, tl, j, u)));
                }
            }
        }
    }
    cp_wait<0>();  // nothing in flight at exit (every staged copy was waited for above)
    if constexpr (TC)
        tc_end(tcx, TCT);
}

// ------------------------------------------------------------------- col_mx
// Zero-rim column pass (forces) with one thread per slot j carrying BOTH
// parity halves of its column: the two forward transforms (x and x W_P^n) run
// as two sequences of one thread, the spectral products of a bin's even and
// odd halves stay in that thread, and the fold y[n] = even[n] + W_P^{-n}
// odd[n] of the inverse transforms is done in registers, so no fold goes
// through shared memory.  The thread keeps its slot for the whole launch (the
// CTA walks the columns), so the twiddles of its slot live in registers
// (load_twiddles_rt) and only the exchanges between stages use shared memory.
// Fy^ waits in registers (or, PARK, in shared memory in slot order) while Fx^
// is transformed back.  The N + 1 columns are shared among G = 256 / (N/16)
// groups of N/16 threads per CTA (one group at N = 4096), each group walking
// its own columns on its own named barrier, with the next column's input and
// spectrum half rows copied in behind the inverse transforms.  FP32, no
// tensor-core tiles, N >= 1024.  NC = 1: the potential of a zero-rim potential
// plan (Gphi, real and even in ky, alone; one inverse transform per column,
// nothing parked).
// Shared memory per group: column[N] | Gx, Gy half rows of both halves |
// exchange buffers [2][SPC] | (PARK) Fy^ [2][N].
// Fy^ parked in shared memory (true) or kept in registers (false).
constexpr bool kMxPark = true;

template <int LOGN, bool PARK>
struct KMx {
    static constexpr int N = 1 << LOGN, Q = N >> 4;
    static constexpr int G = Q >= 256 ? 1 : 256 / Q;
    static constexpr int THREADS = G * Q;
    static constexpr int SPC = col_sp<float2>(N);
    static constexpr size_t GROUP_BYTES = (size_t)N * 8 + 4 * (size_t)quarter_half(N) * 4 + 2 * (size_t)SPC * 8 +
                                          (PARK ? 2 * (size_t)N * 8 : 0);
    static constexpr size_t SMEM = G * GROUP_BYTES;
};

template <int LOGN, bool PARK, int PLAN, int NC = 2>
__global__ void __launch_bounds__(KMx<LOGN, PARK>::THREADS, 1) k_col_mx(SolveArgs<float> a)
{
    constexpr bool two = NC == 2;  // the forces (Gx, Gy); else the potential (Gphi alone)
    using C = float2;
    using M = KMx<LOGN, PARK>;
    using P = FR<LOGN, PLAN>;
    constexpr int N = M::N, Q = M::Q, G = M::G, HQ = quarter_half(N), QS = quarter_stride(N), SPC = M::SPC;
    static_assert(Q >= 64, "named group barriers need whole warps");
    extern __shared__ __align__(16) unsigned char smem_mx[];
    const int t = threadIdx.x;
    const int g = t / Q, j = t - g * Q;
    unsigned char *gbase = smem_mx + (size_t)g * M::GROUP_BYTES;
    C *col = reinterpret_cast<C *>(gbase);
    float *gsp = reinterpret_cast<float *>(col + N);  // [half][Gx, Gy][HQ]
    C *xb = reinterpret_cast<C *>(gbase + (size_t)N * 8 + 4 * (size_t)HQ * 4);
    C *park = xb + 2 * SPC;
    const unsigned bar = 1 + g;
    C trw[P::NST - 1][15];
    load_twiddles_rt<C, LOGN, PLAN>(trw, a.twn, j);
    const TwLayout tl = tw_layout(F16<LOGN>::twlen, N);
    const C wj = a.tw[tl.base + j];  // W_P^j
    auto twist_u = [&](int u) { return hmul(wj, hmk<C>((float)kW32c[u], (float)-kW32s[u])); };
    const float *spec = reinterpret_cast<const float *>(a.spec);
    auto stage = [&](int kx) {  // this group's threads: column kx and its four spectrum half rows
        const char *src = reinterpret_cast<const char *>(a.fwd + (size_t)kx * N);
        for (int o = j * 16; o < N * 8; o += Q * 16)
            cp16(reinterpret_cast<char *>(col) + o, src + o);
        for (int h = 0; h < 4; h += two ? 1 : 2) {  // [half][table]: Gx rows at kx, Gy rows at N + 1 + kx
            const float *row = spec + ((size_t)(h & 1) * (N + 1) + kx) * QS + (h >> 1) * HQ;
            for (int o = j * 16; o < HQ * 4; o += Q * 16)
                cp16(reinterpret_cast<char *>(gsp + h * HQ) + o, reinterpret_cast<const char *>(row) + o);
        }
        cp_commit();
    };
    const int step = (int)gridDim.x * G;
    int kx = (int)blockIdx.x * G + g;
    if (kx <= N)
        stage(kx);
    for (; kx <= N; kx += step) {  // uniform over the group
        cp_wait<0>();
        group_sync(bar, Q);  // column kx staged; the previous column's exchanges are done
        C v[2][16];
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const C x = col[j + u * Q];
            v[0][u] = x;
            v[1][u] = hmul(x, twist_u(u));
        }
        fft_stages_rt<C, false, LOGN, PLAN, 2, 0>(v, xb, SPC, j, trw, bar, Q);
        C fy[PARK || !two ? 1 : 2][16];
        if constexpr (two) {
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                const float *gx_r = gsp + (2 * b) * HQ, *gy_r = gsp + (2 * b + 1) * HQ;
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    const int kp = j + u * Q;
                    const bool hi = 2 * kp + b > N;
                    const int q = hi ? N - kp - b : kp;
                    const float gx = gx_r[q];                  // Gx even in ky
                    const float gy = hi ? -gy_r[q] : gy_r[q];  // Gy odd in ky
                    const C y = hmk<C>(-gy * v[b][u].y, gy * v[b][u].x);  // i gy v
                    if constexpr (PARK)
                        park[b * N + kp] = y;
                    else
                        fy[b][u] = y;
                    v[b][u] = hmk<C>(-gx * v[b][u].y, gx * v[b][u].x);  // i gx v
                }
            }
        } else {
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                const float *gp_r = gsp + (2 * b) * HQ;
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    const int kp = j + u * Q;
                    const int q = 2 * kp + b > N ? N - kp - b : kp;
                    const float gp = gp_r[q];  // Gphi real, even in ky
                    v[b][u] = hmk<C>(gp * v[b][u].x, gp * v[b][u].y);
                }
            }
        }
        if (kx + step <= N) {  // uniform over the group
            group_sync(bar, Q);  // every thread of the group is done with the column and the half rows
            stage(kx + step);
        }
        C *dst = a.bwd;
        fft_stages_rt<C, true, LOGN, PLAN, 2, 0>(v, xb, SPC, j, trw, bar, Q);
#pragma unroll
        for (int u = 0; u < 16; ++u)
            dst[bwd_index(N, N, 0, kx, j + u * Q)] = hadd(v[0][u], hmulc(v[1][u], twist_u(u)));
        if constexpr (two && PARK) {  // Fy^: this thread's own values, no barrier
#pragma unroll
            for (int b = 0; b < 2; ++b)
#pragma unroll
                for (int u = 0; u < 16; ++u)
                    v[b][u] = park[b * N + j + u * Q];
            fft_stages_rt<C, true, LOGN, PLAN, 2, 0>(v, xb, SPC, j, trw, bar, Q);
#pragma unroll
            for (int u = 0; u < 16; ++u)
                dst[bwd_index(N, N, 1, kx, j + u * Q)] = hadd(v[0][u], hmulc(v[1][u], twist_u(u)));
        } else if constexpr (two) {
            fft_stages_rt<C, true, LOGN, PLAN, 2, 0>(fy, xb, SPC, j, trw, bar, Q);
#pragma unroll
            for (int u = 0; u < 16; ++u)
                dst[bwd_index(N, N, 1, kx, j + u * Q)] = hadd(fy[0][u], hmulc(fy[1][u], twist_u(u)));
        }
    }
    cp_wait<0>();  // nothing in flight at exit
}

// ---------------------------------------------------------------- launching
// Dynamic shared memory per kernel; TC adds the tensor-core area in front.
template <typename T, int LOGN, bool TC = false>
struct KSmem {
    using C = typename Cx<T>::C;
    static constexpr int N = 1 << LOGN;
    static size_t tc(int threads, int B, int kind)
    {
        return TC ? tc_smem_bytes(tc_round(LOGN, tc_tiles(threads, B), kind)) : 0;
    }
    static size_t rtc(int kind) { return tc(KShape<LOGN>::ROW_THREADS, 1, kind); }
    static size_t ctc(int kind) { return tc(KShape<LOGN>::COL_THREADS, 2, kind); }
    static size_t tw() { return tw_bytes<C>(tw_layout(F16<LOGN>::twlen, N).entries); }
    static size_t row_fwd()
    {
        // the staged rows (at most 4 N reals) fit in the exchange buffers' 2 SP_ROW complex
        return rtc(KK_ROW_FWD) + tw() + 2 * (size_t)KShape<LOGN>::SP_ROW * sizeof(C);
    }
    static size_t col()
    {
        return ctc(KK_COL) + tw() + (size_t)col_sp<C>(N) * sizeof(C) + 2 * ColStage<T, LOGN, TC>::BYTES;
    }
    static size_t col_w() { return tw() + 2 * (size_t)col_sp<C>(N) * sizeof(C) + 2 * ColWStage<T, LOGN>::BYTES; }
    static size_t row_inv()
    {
        return rtc(KK_ROW_INV) + tw() + ((2 * (size_t)(N + 1) * sizeof(C) + 15) & ~(size_t)15) +
               2 * (size_t)KShape<LOGN>::SP_ROW * sizeof(C) + 4 * (size_t)N * sizeof(T);
    }
    static size_t row_inv1(int nc)
    {
        const size_t stage = (size_t)nc * 2 * (N / 2 + 1) * 2 * sizeof(C);  // [comp][parity][N/2 + 1] pairs
        const size_t xbuf = (size_t)nc * 2 * KShape<LOGN>::SP_ROW * sizeof(C);
        return tc(KShape<LOGN>::ROW_THREADS, nc, nc == 1 ? KK_ROW_INV1 : KK_ROW_INV2) + tw() +
               (stage > xbuf ? stage : xbuf);
    }
    static size_t row_inv1t() { return row_inv1t_body<T, LOGN>() + tw() + 16 + 128; }  // + mbarrier, alignment slack
    static size_t row_fwd_m()
    {
        return rtc(KK_ROW_FWD_M) + tw() + 2 * (size_t)N * sizeof(T) + 2 * (size_t)KShape<LOGN>::SP_ROW * sizeof(C);
    }
    static size_t col_m()
    {
        return tc(KShape<LOGN>::COL_THREADS, 1, KK_COL_M) + tw() + (size_t)col_sp<C>(N) * sizeof(C) +
               (size_t)N * sizeof(C);
    }
    static size_t col_gw()
    {
        return tw() + 4 * (size_t)col_sp<C>(N) * sizeof(C) + 6 * (size_t)N * sizeof(C);
    }
    static size_t col_g()
    {
        return tc(KShape<LOGN>::COL_THREADS, 2, KK_COL_G) + tw() + 2 * (size_t)col_sp<C>(N) * sizeof(C) +
               3 * (size_t)N * sizeof(C);
    }
    static size_t col_sum()
    {
        size_t body = 2 * (size_t)col_sp<C>(N) * sizeof(C);  // two exchange buffers; the 2N fold fits
        return ctc(KK_COL_SUM) + tw() + body;
    }
    static size_t col_mw()
    {
        return tc(KShape<LOGN>::ROW_THREADS, 2, KK_COL_MW) + tw() + (size_t)N * sizeof(C) +
               4 * (size_t)quarter_half(N) * sizeof(T) + 4 * (size_t)col_sp<C>(N) * sizeof(C);
    }
    static size_t col_md()
    {
        // sbuf + column + spectrum half rows; at least two exchange buffers (dual inverse) and the 2N fold
        size_t body = (size_t)col_sp<C>(N) * sizeof(C) + (size_t)N * sizeof(C) + 2 * (size_t)quarter_half(N) * sizeof(T);
        const size_t need = 2 * (size_t)col_sp<C>(N) * sizeof(C);
        if (body < need)
            body = need;
        if (body < 2 * (size_t)N * sizeof(C))
            body = 2 * (size_t)N * sizeof(C);
        return ctc(KK_COL_MD) + tw() + body;
    }
};

// Sets the dynamic shared-memory limit of a kernel once per device.  A kernel
// that needs more than an SM offers (k_row_inv with tensor-core tiles at
// n = 4096, a configuration the host refuses) is left alone here; launching it
// would fail with a launch error.
template <typename F>
inline cudaError_t ensure_smem(F *kernel, size_t bytes, std::atomic<unsigned long long> &done)
{
    if (bytes > kMaxDynSmem)
        return cudaSuccess;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (done.load(std::memory_order_acquire) & bit)
        return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess)
        done.fetch_or(bit, std::memory_order_acq_rel);
    return e;
}

// CTAs of a kernel that are resident on the current device at once (SMs x
// CTAs per SM at this block size and shared memory), found once per device
// for each kernel instance; the grid of a kernel that walks its work items.
template <typename F>
inline cudaError_t resident_ctas(F *kernel, int threads, size_t smem, std::atomic<int> (&cache)[64], int *out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    int n = cache[dev & 63].load(std::memory_order_acquire);
    if (n <= 0) {
        int sms = 0, per_sm = 0;
        if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
            (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem)) != cudaSuccess)
            return e;
        n = sms * (per_sm > 0 ? per_sm : 1);
        cache[dev & 63].store(n, std::memory_order_release);
    }
    *out = n;
    return cudaSuccess;
}

// Grid x of a walking kernel over `items` work items per patch, `count`
// patches side by side in y: the resident CTAs shared among the patches.
inline int min_grid(int items, int resident, int count)
{
    const int per = resident / (count > 0 ? count : 1);
    return per < 1 ? 1 : (per < items ? per : items);
}

template <typename T, int LOGN, bool TC>
cudaError_t launch_pass(int pass, const SolveArgs<T> &a, int count, cudaStream_t st, const BatchView<T> *bv)
{
    using K = KShape<LOGN>;
    using S = KSmem<T, LOGN, TC>;
    static std::atomic<unsigned long long> d[40];
    static std::atomic<int> res_mx[64], res_mx1[64];  // resident CTAs of the register-twiddle column pass (plans 0, 1)
    static std::atomic<int> res_rx[64], res_rx1[64];  // and of the register-twiddle inverse row pass
    static std::atomic<int> res_r2[64], res_r21[64];  // and of its two-pair form
    static std::atomic<int> res_fx[64];               // and of the register-twiddle forward row pass
    static std::atomic<int> res_f3x[64];              // and of its three-field form
    static std::atomic<int> res_mxp[64], res_mxp1[64]; // and of the register-twiddle column pass, potential
    static std::atomic<int> res_mw[64], res_mw1[64];  // resident CTAs of the walking column pass (NC = 2, 1)
    static std::atomic<int> res_fm[64];               // and of the walking zero-rim forward row pass
    static std::atomic<int> res_ri1[64], res_ri2[64]; // and of the walking inverse row passes (tensor cores)
    static std::atomic<int> res_cm[64], res_cmd[64];  // and of the walking cluster column passes (tensor cores)
    const BatchView<T> none{nullptr, nullptr};
    const bool batch = bv != nullptr;
    const BatchView<T> v = batch ? *bv : none;
    cudaError_t e = cudaSuccess;
#define SGF_LAUNCH(K0, K1, idx, smem, grid, threads)                                  \
    if (batch) {                                                                      \
        if ((e = ensure_smem(K1, smem, d[idx + 1])) != cudaSuccess)                   \
            return e;                                                                 \
        K1<<<grid, threads, smem, st>>>(a, v);                                        \
    } else {                                                                          \
        if ((e = ensure_smem(K0, smem, d[idx])) != cudaSuccess)                       \
            return e;                                                                 \
        K0<<<grid, threads, smem, st>>>(a, v);                                        \
    }
    if (pass == PASS_PREPARE) {  // every shared-memory limit and resident count, before any graph capture
        if ((e = ensure_smem(k_row_fwd<T, LOGN, false, TC>, S::row_fwd(), d[0])) != cudaSuccess ||
            (e = ensure_smem(k_row_fwd<T, LOGN, true, TC>, S::row_fwd(), d[1])) != cudaSuccess ||
            (e = ensure_smem(k_col<T, LOGN, false, TC>, S::col(), d[2])) != cudaSuccess ||
            (e = ensure_smem(k_col<T, LOGN, true, TC>, S::col(), d[3])) != cudaSuccess ||
            (e = ensure_smem(k_row_inv<T, LOGN, false, TC>, S::row_inv(), d[4])) != cudaSuccess ||
            (e = ensure_smem(k_row_inv<T, LOGN, true, TC>, S::row_inv(), d[5])) != cudaSuccess ||
            (e = ensure_smem(k_row_fwd_m<T, LOGN, false, TC>, S::row_fwd_m(), d[6])) != cudaSuccess ||
            (e = ensure_smem(k_row_fwd_m<T, LOGN, true, TC>, S::row_fwd_m(), d[7])) != cudaSuccess ||
            (e = ensure_smem(k_col_m<T, LOGN, false, TC>, S::col_m(), d[8])) != cudaSuccess ||
            (e = ensure_smem(k_col_m<T, LOGN, true, TC>, S::col_m(), d[9])) != cudaSuccess ||
            (e = ensure_smem(k_row_inv1<T, LOGN, false, TC, 1>, S::row_inv1(1), d[10])) != cudaSuccess ||
            (e = ensure_smem(k_row_inv1<T, LOGN, true, TC, 1>, S::row_inv1(1), d[11])) != cudaSuccess ||
            (e = ensure_smem(k_row_inv1<T, LOGN, false, TC, 2>, S::row_inv1(2), d[18])) != cudaSuccess ||
            (e = ensure_smem(k_row_inv1<T, LOGN, true, TC, 2>, S::row_inv1(2), d[19])) != cudaSuccess ||
            (e = ensure_smem(k_col_mw<T, LOGN, false, TC>, S::col_mw(), d[20])) != cudaSuccess ||
            (e = ensure_smem(k_col_mw<T, LOGN, true, TC>, S::col_mw(), d[21])) != cudaSuccess ||
            (e = ensure_smem(k_col_md<T, LOGN, false, TC>, S::col_md(), d[12])) != cudaSuccess ||
            (e = ensure_smem(k_col_md<T, LOGN, true, TC>, S::col_md(), d[13])) != cudaSuccess ||
            (e = ensure_smem(k_col_g<T, LOGN, false, TC>, S::col_g(), d[14])) != cudaSuccess ||
            (e = ensure_smem(k_col_g<T, LOGN, true, TC>, S::col_g(), d[15])) != cudaSuccess ||
            (e = ensure_smem(k_col_sum<T, LOGN, false, TC>, S::col_sum(), d[16])) != cudaSuccess ||
            (e = ensure_smem(k_col_sum<T, LOGN, true, TC>, S::col_sum(), d[17])) != cudaSuccess ||
            (e = ensure_smem(k_col_mw<T, LOGN, false, TC, 1>, S::col_mw(), d[25])) != cudaSuccess)
            return e;
        int grid = 0;
        if (S::col_mw() <= kMaxDynSmem &&
            ((e = resident_ctas(k_col_mw<T, LOGN, false, TC>, K::ROW_THREADS, S::col_mw(), res_mw, &grid)) !=
                 cudaSuccess ||
             (e = resident_ctas(k_col_mw<T, LOGN, false, TC, 1>, K::ROW_THREADS, S::col_mw(), res_mw1, &grid)) !=
                 cudaSuccess))
            return e;
        if (S::row_fwd_m() <= kMaxDynSmem &&
            (e = resident_ctas(k_row_fwd_m<T, LOGN, false, TC>, K::ROW_THREADS, S::row_fwd_m(), res_fm, &grid)) !=
                cudaSuccess)
            return e;
        if constexpr (TC) {  // the walking tensor-core instances
            if ((S::row_inv1(1) <= kMaxDynSmem &&
                 (e = resident_ctas(k_row_inv1<T, LOGN, false, TC, 1>, K::ROW_THREADS, S::row_inv1(1), res_ri1,
                                    &grid)) != cudaSuccess) ||
                (S::row_inv1(2) <= kMaxDynSmem &&
                 (e = resident_ctas(k_row_inv1<T, LOGN, false, TC, 2>, K::ROW_THREADS, S::row_inv1(2), res_ri2,
                                    &grid)) != cudaSuccess) ||
                (S::col_m() <= kMaxDynSmem &&
                 (e = resident_ctas(k_col_m<T, LOGN, false, TC>, K::COL_THREADS, S::col_m(), res_cm, &grid)) !=
                     cudaSuccess) ||
                (S::col_md() <= kMaxDynSmem &&
                 (e = resident_ctas(k_col_md<T, LOGN, false, TC>, K::COL_THREADS, S::col_md(), res_cmd, &grid)) !=
                     cudaSuccess))
                return e;
        }
        if constexpr (!TC && K::HB_ROW > 0 && sizeof(T) == 4) {  // the FP32-only kernels
            if ((S::col_w() <= kMaxDynSmem &&
                 ((e = ensure_smem(k_col_w<T, LOGN, false>, S::col_w(), d[23])) != cudaSuccess ||
                  (e = ensure_smem(k_col_w<T, LOGN, true>, S::col_w(), d[24])) != cudaSuccess)) ||
                (S::col_gw() <= kMaxDynSmem &&
                 ((e = ensure_smem(k_col_gw<T, LOGN, false>, S::col_gw(), d[26])) != cudaSuccess ||
                  (e = ensure_smem(k_col_gw<T, LOGN, true>, S::col_gw(), d[27])) != cudaSuccess)) ||
                (e = ensure_smem(k_row_inv1t<T, LOGN>, S::row_inv1t(), d[22])) != cudaSuccess)
                return e;
        }
        if constexpr (!TC && sizeof(T) == 4 && LOGN >= 10) {
            using MX = KMx<LOGN, kMxPark>;
            using RX = KRx<LOGN>;
            if ((e = ensure_smem(k_col_mx<LOGN, kMxPark, 0>, MX::SMEM, d[28])) != cudaSuccess ||
                (e = resident_ctas(k_col_mx<LOGN, kMxPark, 0>, MX::THREADS, MX::SMEM, res_mx, &grid)) != cudaSuccess ||
                (e = ensure_smem(k_col_mx<LOGN, kMxPark, 1>, MX::SMEM, d[30])) != cudaSuccess ||
                (e = resident_ctas(k_col_mx<LOGN, kMxPark, 1>, MX::THREADS, MX::SMEM, res_mx1, &grid)) != cudaSuccess ||
                (e = ensure_smem(k_row_inv1x<LOGN, 0>, RX::SMEM, d[29])) != cudaSuccess ||
                (e = resident_ctas(k_row_inv1x<LOGN, 0>, RX::THREADS, RX::SMEM, res_rx, &grid)) != cudaSuccess ||
                (e = ensure_smem(k_row_inv1x<LOGN, 1>, RX::SMEM, d[31])) != cudaSuccess ||
                (e = resident_ctas(k_row_inv1x<LOGN, 1>, RX::THREADS, RX::SMEM, res_rx1, &grid)) != cudaSuccess ||
                (e = ensure_smem(k_row_inv2x<LOGN, 0>, KR2x<LOGN>::SMEM, d[33])) != cudaSuccess ||
                (e = resident_ctas(k_row_inv2x<LOGN, 0>, KR2x<LOGN>::THREADS, KR2x<LOGN>::SMEM, res_r2, &grid)) !=
                    cudaSuccess ||
                (e = ensure_smem(k_row_inv2x<LOGN, 1>, KR2x<LOGN>::SMEM, d[34])) != cudaSuccess ||
                (e = ensure_smem(k_row_fwd2<LOGN>, S::tw() + 4 * (size_t)K::SP_ROW * sizeof(float2), d[35])) !=
                    cudaSuccess ||
                (e = ensure_smem(k_row_fwd_x<LOGN, 0>, KFx<LOGN>::SMEM, d[36])) != cudaSuccess ||
                (e = ensure_smem(k_row_fwd3x<LOGN, 0>, KF3x<LOGN>::SMEM, d[39])) != cudaSuccess ||
                (e = resident_ctas(k_row_fwd3x<LOGN, 0>, KF3x<LOGN>::THREADS, KF3x<LOGN>::SMEM, res_f3x, &grid)) !=
                    cudaSuccess ||
                (e = ensure_smem(k_col_mx<LOGN, kMxPark, 0, 1>, MX::SMEM, d[37])) != cudaSuccess ||
                (e = resident_ctas(k_col_mx<LOGN, kMxPark, 0, 1>, MX::THREADS, MX::SMEM, res_mxp, &grid)) !=
                    cudaSuccess ||
                (e = ensure_smem(k_col_mx<LOGN, kMxPark, 1, 1>, MX::SMEM, d[38])) != cudaSuccess ||
                (e = resident_ctas(k_col_mx<LOGN, kMxPark, 1, 1>, MX::THREADS, MX::SMEM, res_mxp1, &grid)) !=
                    cudaSuccess ||
                (e = resident_ctas(k_row_fwd_x<LOGN, 0>, KFx<LOGN>::THREADS, KFx<LOGN>::SMEM, res_fx, &grid)) !=
                    cudaSuccess ||
                (e = resident_ctas(k_row_inv2x<LOGN, 1>, KR2x<LOGN>::THREADS, KR2x<LOGN>::SMEM, res_r21, &grid)) !=
                    cudaSuccess ||
                (e = ensure_smem(k_row_fwd_m2<LOGN>, S::tw() + 4 * (size_t)K::N * sizeof(float) +
                                                         4 * (size_t)K::SP_ROW * sizeof(float2), d[32])) != cudaSuccess)
                return e;
        }
        return cudaSuccess;
    }
    switch (pass) {
    case PASS_ROW_FWD: {
        SGF_LAUNCH((k_row_fwd<T, LOGN, false, TC>), (k_row_fwd<T, LOGN, true, TC>), 0, S::row_fwd(), dim3(count, 3),
                   K::ROW_THREADS)
        break;
    }
    case PASS_COL: {
        // tensor-core tiles: each cluster walks kColWalk columns of its work item (strided by the
        // clusters of the item), which keeps many clusters per item for balance
        const int gx = TC && !batch ? 2 * ((K::N + 1 + kColWalk - 1) / kColWalk) : 2 * (K::N + 1);
        SGF_LAUNCH((k_col<T, LOGN, false, TC>), (k_col<T, LOGN, true, TC>), 2, S::col(), dim3(gx, count),
                   K::COL_THREADS)
        break;
    }
    case PASS_ROW_INV: {
        SGF_LAUNCH((k_row_inv<T, LOGN, false, TC>), (k_row_inv<T, LOGN, true, TC>), 4, S::row_inv(), dim3(K::N / 2, count),
                   K::ROW_THREADS)
        break;
    }
    case PASS_ROW_INV1: {
        // tensor-core tiles: the CTAs that fit at once (over the count patches) walk the row pairs
        int gx = batch ? K::N : a.ncomp * (K::N / 2);
        if (TC && !batch) {
            int res = 0;
            if ((e = ensure_smem(k_row_inv1<T, LOGN, false, TC, 1>, S::row_inv1(1), d[10])) != cudaSuccess ||
                (e = resident_ctas(k_row_inv1<T, LOGN, false, TC, 1>, K::ROW_THREADS, S::row_inv1(1), res_ri1,
                                   &res)) != cudaSuccess)
                return e;
            gx = min_grid(gx, res, count);
        }
        SGF_LAUNCH((k_row_inv1<T, LOGN, false, TC, 1>), (k_row_inv1<T, LOGN, true, TC, 1>), 10, S::row_inv1(1),
                   dim3(gx, count), K::ROW_THREADS)
        break;
    }
    case PASS_ROW_INV2: {
        int gx = K::N / 2;
        if (TC && !batch) {
            int res = 0;
            if ((e = ensure_smem(k_row_inv1<T, LOGN, false, TC, 2>, S::row_inv1(2), d[18])) != cudaSuccess ||
                (e = resident_ctas(k_row_inv1<T, LOGN, false, TC, 2>, K::ROW_THREADS, S::row_inv1(2), res_ri2,
                                   &res)) != cudaSuccess)
                return e;
            gx = min_grid(gx, res, count);
        }
        SGF_LAUNCH((k_row_inv1<T, LOGN, false, TC, 2>), (k_row_inv1<T, LOGN, true, TC, 2>), 18, S::row_inv1(2),
                   dim3(gx, count), K::ROW_THREADS)
        break;
    }
    case PASS_ROW_FWD_M: {
        // tensor-core tiles: the CTAs that fit at once walk the N / 2 row pairs (one tensor-memory
        // allocation per CTA); otherwise, and in batches, one CTA per (pair, item), which measured faster
        int grid = K::N / 2;
        if (TC && !batch && ((e = ensure_smem(k_row_fwd_m<T, LOGN, false, TC>, S::row_fwd_m(), d[6])) != cudaSuccess ||
                       (e = resident_ctas(k_row_fwd_m<T, LOGN, false, TC>, K::ROW_THREADS, S::row_fwd_m(), res_fm,
                                          &grid)) != cudaSuccess))
            return e;
        SGF_LAUNCH((k_row_fwd_m<T, LOGN, false, TC>), (k_row_fwd_m<T, LOGN, true, TC>), 6, S::row_fwd_m(),
                   dim3(grid < K::N / 2 ? grid : K::N / 2, batch ? count : 1), K::ROW_THREADS)
        break;
    }
    case PASS_COL_M: {
        // tensor-core tiles: the 2-CTA clusters that fit at once walk the N + 1 columns
        int gx = 2 * (K::N + 1);
        if (TC && !batch) {
            int res = 0;
            if ((e = ensure_smem(k_col_m<T, LOGN, false, TC>, S::col_m(), d[8])) != cudaSuccess ||
                (e = resident_ctas(k_col_m<T, LOGN, false, TC>, K::COL_THREADS, S::col_m(), res_cm, &res)) !=
                    cudaSuccess)
                return e;
            gx = 2 * min_grid(K::N + 1, res / 2, 1);
        }
        SGF_LAUNCH((k_col_m<T, LOGN, false, TC>), (k_col_m<T, LOGN, true, TC>), 8, S::col_m(),
                   dim3(gx, batch ? count : 1), K::COL_THREADS)
        break;
    }
    case PASS_COL_SUM: {
        SGF_LAUNCH((k_col_sum<T, LOGN, false, TC>), (k_col_sum<T, LOGN, true, TC>), 16, S::col_sum(),
                   dim3(2 * (K::N + 1), count), K::COL_THREADS)
        break;
    }
    case PASS_COL_G: {
        SGF_LAUNCH((k_col_g<T, LOGN, false, TC>), (k_col_g<T, LOGN, true, TC>), 14, S::col_g(),
                   dim3(2 * (K::N + 1), count), K::COL_THREADS)
        break;
    }
    case PASS_COL_MW: {
        // one pass: the CTAs that fit at once walk the N + 1 columns; batches: one CTA per (column, item)
        int grid = 0;
        if (!batch && a.ncomp == 1) {  // the zero-rim potential (plans of one patch; never batched)
            if ((e = ensure_smem(k_col_mw<T, LOGN, false, TC, 1>, S::col_mw(), d[25])) != cudaSuccess ||
                (e = resident_ctas(k_col_mw<T, LOGN, false, TC, 1>, K::ROW_THREADS, S::col_mw(), res_mw1, &grid)) !=
                    cudaSuccess)
                return e;
            k_col_mw<T, LOGN, false, TC, 1><<<dim3(grid < K::N + 1 ? grid : K::N + 1, 1), K::ROW_THREADS,
                                               S::col_mw(), st>>>(a, v);
            break;
        }
        if (batch) {
            grid = K::N + 1;
        } else if ((e = ensure_smem(k_col_mw<T, LOGN, false, TC>, S::col_mw(), d[20])) != cudaSuccess ||
                   (e = resident_ctas(k_col_mw<T, LOGN, false, TC>, K::ROW_THREADS, S::col_mw(), res_mw, &grid)) !=
                       cudaSuccess) {
            return e;
        }
        SGF_LAUNCH((k_col_mw<T, LOGN, false, TC>), (k_col_mw<T, LOGN, true, TC>), 20, S::col_mw(),
                   dim3(grid < K::N + 1 ? grid : K::N + 1, batch ? count : 1), K::ROW_THREADS)
        break;
    }
    case PASS_COL_W: {
        if constexpr (!TC && K::HB_ROW > 0 && sizeof(T) == 4) {  // FP64's two sequences need > 128 registers
            if (S::col_w() > kMaxDynSmem)
                return cudaErrorInvalidConfiguration;
            SGF_LAUNCH((k_col_w<T, LOGN, false>), (k_col_w<T, LOGN, true>), 23, S::col_w(),
                       batch ? dim3(count, K::N + 1) : dim3(K::N + 1, count), K::ROW_THREADS)
        } else {
            return cudaErrorInvalidValue;
        }
        break;
    }
    case PASS_COL_GW: {
        if constexpr (!TC && K::HB_ROW > 0 && sizeof(T) == 4) {
            if (S::col_gw() > kMaxDynSmem)
                return cudaErrorInvalidConfiguration;
            SGF_LAUNCH((k_col_gw<T, LOGN, false>), (k_col_gw<T, LOGN, true>), 26, S::col_gw(),
                       dim3(K::N + 1, count), K::ROW_THREADS)
        } else {
            return cudaErrorInvalidValue;
        }
        break;
    }
    case PASS_ROW_INV1T: {
        if constexpr (sizeof(T) == 4 && !TC && K::HB_ROW > 0) {
            if (batch)
                return cudaErrorInvalidValue;
            if ((e = ensure_smem(k_row_inv1t<T, LOGN>, S::row_inv1t(), d[22])) != cudaSuccess)
                return e;
            k_row_inv1t<T, LOGN><<<dim3(a.ncomp * (K::N / 2), count), K::ROW_THREADS, S::row_inv1t(), st>>>(a);
        } else {
            return cudaErrorInvalidValue;
        }
        break;
    }
    case PASS_ROW_INV1X:
    case PASS_ROW_INV1X_R1: {
        if constexpr (!TC && sizeof(T) == 4 && LOGN >= 10) {
            if (batch)
                return cudaErrorInvalidValue;
            using RX = KRx<LOGN>;
            const bool r1 = pass == PASS_ROW_INV1X_R1;
            auto *kern = r1 ? k_row_inv1x<LOGN, 1> : k_row_inv1x<LOGN, 0>;
            int grid = 0;
            if ((e = ensure_smem(kern, RX::SMEM, d[r1 ? 31 : 29])) != cudaSuccess ||
                (e = resident_ctas(kern, RX::THREADS, RX::SMEM, r1 ? res_rx1 : res_rx, &grid)) != cudaSuccess)
                return e;
            const int groups = (a.ncomp * (K::N / 2) + RX::G - 1) / RX::G;  // CTAs that give every group an item
            kern<<<dim3(grid < groups ? grid : groups, count), RX::THREADS, RX::SMEM, st>>>(a);
        } else {
            return cudaErrorInvalidValue;
        }
        break;
    }
    case PASS_ROW_INV2X:
    case PASS_ROW_INV2X_R1: {
        if constexpr (!TC && sizeof(T) == 4 && LOGN >= 10) {
            if (batch)
                return cudaErrorInvalidValue;
            using R2 = KR2x<LOGN>;
            const bool r1 = pass == PASS_ROW_INV2X_R1;
            auto *kern = r1 ? k_row_inv2x<LOGN, 1> : k_row_inv2x<LOGN, 0>;
            int grid = 0;
            if ((e = ensure_smem(kern, R2::SMEM, d[r1 ? 34 : 33])) != cudaSuccess ||
                (e = resident_ctas(kern, R2::THREADS, R2::SMEM, r1 ? res_r21 : res_r2, &grid)) != cudaSuccess)
                return e;
            const int groups = (a.ncomp * (K::N / 4) + R2::G - 1) / R2::G;  // CTAs that give every group an item
            kern<<<dim3(grid < groups ? grid : groups, count), R2::THREADS, R2::SMEM, st>>>(a);
        } else {
            return cudaErrorInvalidValue;
        }
        break;
    }
    case PASS_ROW_FWD3X: {
        if constexpr (!TC && sizeof(T) == 4 && LOGN >= 10) {
            if (batch)
                return cudaErrorInvalidValue;
            using F3 = KF3x<LOGN>;
            int grid = 0;
            if ((e = ensure_smem(k_row_fwd3x<LOGN, 0>, F3::SMEM, d[39])) != cudaSuccess ||
                (e = resident_ctas(k_row_fwd3x<LOGN, 0>, F3::THREADS, F3::SMEM, res_f3x, &grid)) != cudaSuccess)
                return e;
            const int groups = (K::N / 2 + F3::G - 1) / F3::G;  // CTAs that give every group a row pair
            k_row_fwd3x<LOGN, 0><<<grid < groups ? grid : groups, F3::THREADS, F3::SMEM, st>>>(a);
        } else {
            return cudaErrorInvalidValue;
        }
        break;
    }
    case PASS_ROW_FWD_X: {
        if constexpr (!TC && sizeof(T) == 4 && LOGN >= 10) {
            if (batch)
                return cudaErrorInvalidValue;
            using FX = KFx<LOGN>;
            int grid = 0;
            if ((e = ensure_smem(k_row_fwd_x<LOGN, 0>, FX::SMEM, d[36])) != cudaSuccess ||
                (e = resident_ctas(k_row_fwd_x<LOGN, 0>, FX::THREADS, FX::SMEM, res_fx, &grid)) != cudaSuccess)
                return e;
            const int groups = (K::N / 4 + FX::G - 1) / FX::G;  // CTAs that give every group an item
            k_row_fwd_x<LOGN, 0><<<grid < groups ? grid : groups, FX::THREADS, FX::SMEM, st>>>(a);
        } else {
            return cudaErrorInvalidValue;
        }
        break;
    }
    case PASS_ROW_FWD2: {
        if constexpr (!TC && sizeof(T) == 4 && LOGN >= 10) {
            if (batch)
                return cudaErrorInvalidValue;
            const size_t smem = S::tw() + 4 * (size_t)K::SP_ROW * sizeof(float2);
            if ((e = ensure_smem(k_row_fwd2<LOGN>, smem, d[35])) != cudaSuccess)
                return e;
            if (count > 0)
                k_row_fwd2<LOGN><<<(count + 1) / 2, K::N / 4, smem, st>>>(a, count);
        } else {
            return cudaErrorInvalidValue;
        }
        break;
    }
    case PASS_ROW_FWD_M2: {
        if constexpr (!TC && sizeof(T) == 4 && LOGN >= 10) {
            if (batch)
                return cudaErrorInvalidValue;
            const size_t smem = S::tw() + 4 * (size_t)K::N * sizeof(float) + 4 * (size_t)K::SP_ROW * sizeof(float2);
            if ((e = ensure_smem(k_row_fwd_m2<LOGN>, smem, d[32])) != cudaSuccess)
                return e;
            k_row_fwd_m2<LOGN><<<K::N / 4, K::N / 4, smem, st>>>(a);
        } else {
            return cudaErrorInvalidValue;
        }
        break;
    }
    case PASS_COL_MX:
    case PASS_COL_MX_R1: {
        if constexpr (!TC && sizeof(T) == 4 && LOGN >= 10) {
            if (batch)
                return cudaErrorInvalidValue;
            using MX = KMx<LOGN, kMxPark>;
            const bool r1 = pass == PASS_COL_MX_R1;
            const bool pot = a.ncomp == 1;  // the zero-rim potential
            auto *kern = pot ? (r1 ? k_col_mx<LOGN, kMxPark, 1, 1> : k_col_mx<LOGN, kMxPark, 0, 1>)
                             : (r1 ? k_col_mx<LOGN, kMxPark, 1> : k_col_mx<LOGN, kMxPark, 0>);
            int grid = 0;
            if ((e = ensure_smem(kern, MX::SMEM, d[pot ? (r1 ? 38 : 37) : (r1 ? 30 : 28)])) != cudaSuccess ||
                (e = resident_ctas(kern, MX::THREADS, MX::SMEM, pot ? (r1 ? res_mxp1 : res_mxp) : (r1 ? res_mx1 : res_mx),
                                   &grid)) != cudaSuccess)
                return e;
            const int groups = (K::N + 1 + MX::G - 1) / MX::G;  // CTAs that give every group a column
            kern<<<grid < groups ? grid : groups, MX::THREADS, MX::SMEM, st>>>(a);
        } else {
            return cudaErrorInvalidValue;
        }
        break;
    }
    case PASS_COL_MD: {
        int gx = 2 * (K::N + 1);  // as PASS_COL_M
        if (TC && !batch) {
            int res = 0;
            if ((e = ensure_smem(k_col_md<T, LOGN, false, TC>, S::col_md(), d[12])) != cudaSuccess ||
                (e = resident_ctas(k_col_md<T, LOGN, false, TC>, K::COL_THREADS, S::col_md(), res_cmd, &res)) !=
                    cudaSuccess)
                return e;
            gx = 2 * min_grid(K::N + 1, res / 2, 1);
        }
        SGF_LAUNCH((k_col_md<T, LOGN, false, TC>), (k_col_md<T, LOGN, true, TC>), 12, S::col_md(),
                   dim3(gx, batch ? count : 1), K::COL_THREADS)
        break;
    }
    default:
        return cudaErrorInvalidValue;
    }
#undef SGF_LAUNCH
    return cudaGetLastError();
}

}  // namespace sgf
