// sgf_solve.cu -- the per-solve kernels of libsgf.
//
//  restrict : every covered cell of level l takes the mean of its four
//             children on level l+1 (these values only feed the slopes of the
//             uncovered neighbours; covered cells carry no mass).
//  row_fwd  : per source slab and pair of rows, build the three source fields
//             of Eq. (eqnSigma) -- sigma, and the x and y per-cell differences
//             (central inside the patch, one-sided on its first and last
//             cell), zero on covered cells -- gather the slab's phase
//             (Case 2, Eq. eqnbmnn), and transform the rows (real, zero-padded
//             to P = 2N; two real rows travel as one complex row).
//  col      : per output and column kx, transform each input slab's column,
//             multiply by the kernel spectra and accumulate Fx^ and Fy^ for
//             all three fields and all inputs in frequency space (the sums of
//             products of Sec. 2.2), then inverse-transform the column and
//             keep the rows the target needs.
//  row_inv  : per target level and pair of rows, inverse-transform the rows
//             of every output that reaches them (the level's own output and,
//             for every coarser level, its m target phases, Eq. eqnbnmn),
//             interleave the phases into the target cells, zero covered cells
//             and store Fx, Fy.
#include "sgf_fft.cuh"
#include "sgf_internal.h"

namespace sgf {

template <typename T> struct Cpx;
template <> struct Cpx<float> { using C = float2; };
template <> struct Cpx<double> { using C = double2; };

// ------------------------------------------------------------------ restrict
template <typename T>
__global__ void k_restrict(const T *__restrict__ fine, T *__restrict__ coarse,
                           const T *__restrict__ coarse_in, int N, int ox, int oy)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= N * N)
        return;
    const int j = idx / N, i = idx - j * N;
    const int half = N >> 1;
    T v = coarse_in[idx];
    if (i >= ox && i < ox + half && j >= oy && j < oy + half) {
        const int ci = 2 * (i - ox), cj = 2 * (j - oy);
        const T *f = fine + (size_t)cj * N + ci;
        v = T(0.25) * ((f[0] + f[1]) + (f[N] + f[N + 1]));
    }
    coarse[idx] = v;
}

template <typename T>
cudaError_t launch_restrict(const T *fine, T *coarse, const T *coarse_in, int N, int ox, int oy,
                            cudaStream_t st)
{
    const int n = N * N, bs = 256;
    k_restrict<T><<<(n + bs - 1) / bs, bs, 0, st>>>(fine, coarse, coarse_in, N, ox, oy);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ row_fwd
template <typename T>
__device__ __forceinline__ bool is_covered(const SolveArgs<T> &a, int s, int j, int i)
{
    const int ox = a.child_ox[s];
    if (ox < 0)
        return false;
    const int oy = a.child_oy[s], half = a.N >> 1;
    return i >= ox && i < ox + half && j >= oy && j < oy + half;
}

// Field f of level s at cell (j, i): 0 sigma, 1 x difference, 2 y difference.
template <typename T>
__device__ __forceinline__ T field_value(const SolveArgs<T> &a, int s, int j, int i, int f)
{
    if (is_covered(a, s, j, i))
        return T(0);
    const int N = a.N;
    const T *src = a.src[s];
    const T *row = src + (size_t)j * N;
    if (f == 0)
        return row[i];
    if (f == 1) {
        if (i == 0)
            return row[1] - row[0];
        if (i == N - 1)
            return row[N - 1] - row[N - 2];
        return T(0.5) * (row[i + 1] - row[i - 1]);
    }
    if (j == 0)
        return src[(size_t)N + i] - src[i];
    if (j == N - 1)
        return src[(size_t)(N - 1) * N + i] - src[(size_t)(N - 2) * N + i];
    return T(0.5) * (src[(size_t)(j + 1) * N + i] - src[(size_t)(j - 1) * N + i]);
}

template <typename T>
__global__ void k_row_fwd(SolveArgs<T> a)
{
    using C = typename Cpx<T>::C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *W = reinterpret_cast<C *>(smem_raw);  // 2N: parity halves
    const FwdItem item = a.fwd_items[blockIdx.x];
    const FwdSlab sl = a.slabs[item.slab];
    const int N = a.N, tid = threadIdx.x, nt = blockDim.x;
    const int rows = sl.rows, r0 = 2 * item.row_pair;
    const int ja = sl.m * r0 + sl.py, jb = sl.m * (r0 + 1) + sl.py;
    C *out = a.fwd + sl.off;
    for (int f = 0; f < 3; ++f) {
        for (int c = tid; c < N; c += nt) {
            C z = mk<C>(T(0), T(0));
            if (c < rows) {
                const int i = sl.m * c + sl.px;
                z = mk<C>(field_value(a, sl.level, ja, i, f), field_value(a, sl.level, jb, i, f));
            }
            W[c] = z;
            W[N + c] = cmul(z, a.tw[c]);
        }
        __syncthreads();
        block_fft<C, false>(W, N, a.logN, 2, a.tw);
        // unpack the two real rows: X_a = (Z + conj Z~)/2, X_b = (Z - conj Z~)/(2i),
        // Z~ the bin at -kx, which lies in the same parity half
        for (int kx = tid; kx <= N; kx += nt) {
            const int b = kx & 1, k = kx >> 1;
            const int km = (N - b - k) & (N - 1);
            const C Z = W[b * N + k];
            const C Zm = cconj(W[b * N + km]);
            const C s = cadd(Z, Zm), d = csub(Z, Zm);
            const C ya = mk<C>(T(0.5) * s.x, T(0.5) * s.y);
            const C yb = mk<C>(T(0.5) * d.y, T(-0.5) * d.x);
            C *o = out + ((size_t)f * (N + 1) + kx) * rows + r0;
            o[0] = ya;
            o[1] = yb;
        }
        __syncthreads();
    }
}

// --------------------------------------------------------------------- col
template <typename T>
__global__ void k_col(SolveArgs<T> a)
{
    using C = typename Cpx<T>::C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = a.N, P = 2 * N, tid = threadIdx.x, nt = blockDim.x;
    C *W = reinterpret_cast<C *>(smem_raw);  // 2N
    C *AX = W + 2 * N;                       // 2N
    C *AY = AX + 2 * N;                      // 2N
    const int kx = blockIdx.x;
    const ColOutput o = a.outs[blockIdx.y];
    for (int i = tid; i < 2 * N; i += nt) {
        AX[i] = mk<C>(T(0), T(0));
        AY[i] = mk<C>(T(0), T(0));
    }
    for (int in = 0; in < o.in_count; ++in) {
        const ColInput ci = a.ins[o.in_begin + in];
        const FwdSlab sl = a.slabs[ci.slab];
        const int rows = sl.rows;
        for (int f = 0; f < 3; ++f) {
            const C *col = a.fwd + sl.off + ((size_t)f * (N + 1) + kx) * rows;
            for (int n = tid; n < N; n += nt) {
                const C x = n < rows ? col[n] : mk<C>(T(0), T(0));
                W[n] = x;
                W[N + n] = cmul(x, a.tw[n]);
            }
            __syncthreads();
            block_fft<C, false>(W, N, a.logN, 2, a.tw);
            if (ci.kind == SPEC_QUARTER) {
                // tables f (x-force) and 3+f (y-force); K0x, K0y are imaginary,
                // the rest real; mirror sign in ky: + for K0x Kxx Kyy, - for Kxy K0y Kyx
                const T *sx = reinterpret_cast<const T *>(a.spec) + ci.spec_off +
                              ((size_t)f * (N + 1) + kx) * (N + 1);
                const T *sy = reinterpret_cast<const T *>(a.spec) + ci.spec_off +
                              ((size_t)(3 + f) * (N + 1) + kx) * (N + 1);
                const T mx = (f == 2) ? T(-1) : T(1);
                const T my = (f == 2) ? T(1) : T(-1);
                for (int q = tid; q <= N; q += nt) {
                    const T rx = sx[q], ry = sy[q];
                    const int b = q & 1, k1 = q >> 1;
                    const int p1 = b * N + k1;
                    const C X1 = W[p1];
                    C tx = mk<C>(rx * X1.x, rx * X1.y), ty = mk<C>(ry * X1.x, ry * X1.y);
                    if (f == 0) {
                        tx = mk<C>(-tx.y, tx.x);  // times i
                        ty = mk<C>(-ty.y, ty.x);
                    }
                    AX[p1] = cadd(AX[p1], tx);
                    AY[p1] = cadd(AY[p1], ty);
                    if (q != 0 && q != N) {
                        const int p2 = b * N + (N - k1 - b);  // bin P - q
                        const C X2 = W[p2];
                        C ux = mk<C>(mx * rx * X2.x, mx * rx * X2.y);
                        C uy = mk<C>(my * ry * X2.x, my * ry * X2.y);
                        if (f == 0) {
                            ux = mk<C>(-ux.y, ux.x);
                            uy = mk<C>(-uy.y, uy.x);
                        }
                        AX[p2] = cadd(AX[p2], ux);
                        AY[p2] = cadd(AY[p2], uy);
                    }
                }
            } else {
                const C *sx = reinterpret_cast<const C *>(a.spec) + ci.spec_off +
                              ((size_t)f * (N + 1) + kx) * P;
                const C *sy = reinterpret_cast<const C *>(a.spec) + ci.spec_off +
                              ((size_t)(3 + f) * (N + 1) + kx) * P;
                for (int ky = tid; ky < P; ky += nt) {
                    const int p = (ky & 1) * N + (ky >> 1);
                    const C X = W[p];
                    AX[p] = cadd(AX[p], cmul(sx[ky], X));
                    AY[p] = cadd(AY[p], cmul(sy[ky], X));
                }
            }
            __syncthreads();
        }
    }
    block_fft<C, true>(AX, N, a.logN, 2, a.tw);
    block_fft<C, true>(AY, N, a.logN, 2, a.tw);
    // y[n] = even-half[n] + W_P^{-n} odd-half[n] (the 1/P^2 lives in the spectra)
    C *dst = a.bwd + o.off;
    for (int n = tid; n < o.rows; n += nt) {
        const C w = a.tw[n];
        dst[(size_t)kx * o.rows + n] = cadd(AX[n], cmulc(AX[N + n], w));
        dst[((size_t)(N + 1) + kx) * o.rows + n] = cadd(AY[n], cmulc(AY[N + n], w));
    }
}

// ------------------------------------------------------------------ row_inv
template <typename T>
__global__ void k_row_inv(SolveArgs<T> a)
{
    using C = typename Cpx<T>::C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = a.N, P = 2 * N, tid = threadIdx.x, nt = blockDim.x;
    C *W = reinterpret_cast<C *>(smem_raw);            // 2N
    T *O = reinterpret_cast<T *>(W + 2 * N);           // [comp 0..1][row 0..1][N]
    const int t = blockIdx.y;
    const int j0 = 2 * blockIdx.x, j1 = j0 + 1;
    for (int i = tid; i < 4 * N; i += nt)
        O[i] = T(0);
    for (int c = a.contrib_begin[t]; c < a.contrib_begin[t + 1]; ++c) {
        const RowContrib rc = a.contribs[c];
        const ColOutput oa = a.outs[rc.out_base + (j0 % rc.m) * rc.m];
        const ColOutput ob = a.outs[rc.out_base + (j1 % rc.m) * rc.m];
        const int ra = j0 / rc.m, rb = j1 / rc.m;
        const int nout = N / rc.m;
        for (int comp = 0; comp < 2; ++comp) {
            const C *ya = a.bwd + oa.off + (size_t)comp * (N + 1) * oa.rows + ra;
            const C *yb = a.bwd + ob.off + (size_t)comp * (N + 1) * ob.rows + rb;
            // Z[kx] = Ya[kx] + i Yb[kx] over the full period, from the stored half kx <= N
            for (int kk = tid; kk < 2 * N; kk += nt) {
                const int b = kk >= N, k = kk - b * N;
                const int kx = 2 * k + b;
                C z;
                if (kx <= N) {
                    const C A = ya[(size_t)kx * oa.rows], B = yb[(size_t)kx * ob.rows];
                    z = mk<C>(A.x - B.y, A.y + B.x);
                } else {
                    const int k2 = P - kx;
                    const C A = ya[(size_t)k2 * oa.rows], B = yb[(size_t)k2 * ob.rows];
                    z = mk<C>(A.x + B.y, B.x - A.y);  // conj(A) + i conj(B)
                }
                W[kk] = z;
            }
            __syncthreads();
            block_fft<C, true>(W, N, a.logN, 2, a.tw);
            T *Oc = O + comp * 2 * N;
            for (int n = tid; n < nout; n += nt) {
                const C y = cadd(W[n], cmulc(W[N + n], a.tw[n]));
                const int i = rc.m * n + rc.px;
                Oc[i] += y.x;
                Oc[N + i] += y.y;
            }
            __syncthreads();
        }
    }
    T *fx = a.fx[t], *fy = a.fy[t];
    for (int i = tid; i < N; i += nt) {
        const bool ca = is_covered(a, t, j0, i), cb = is_covered(a, t, j1, i);
        fx[(size_t)j0 * N + i] = ca ? T(0) : O[i];
        fx[(size_t)j1 * N + i] = cb ? T(0) : O[N + i];
        fy[(size_t)j0 * N + i] = ca ? T(0) : O[2 * N + i];
        fy[(size_t)j1 * N + i] = cb ? T(0) : O[3 * N + i];
    }
}

// ---------------------------------------------------------------- launchers
static inline int fft_threads(int N, int batch)
{
    // B*N values per block, at most kFftVpt per thread; at least one warp
    int nt = (batch * N) / kFftVpt;
    if (nt < 64)
        nt = 64;
    if (nt > 1024)
        nt = 1024;
    return nt;
}

template <typename T>
size_t smem_col_bytes(int N) { return (size_t)6 * N * sizeof(typename Cpx<T>::C); }
template <typename T>
static size_t smem_row_fwd_bytes(int N) { return (size_t)2 * N * sizeof(typename Cpx<T>::C); }
template <typename T>
static size_t smem_row_inv_bytes(int N) { return (size_t)2 * N * sizeof(typename Cpx<T>::C) + (size_t)4 * N * sizeof(T); }

template <typename T>
cudaError_t solve_kernels_init()
{
    const int maxN = sizeof(T) == 8 ? 2048 : 4096;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_row_fwd<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem_row_fwd_bytes<T>(maxN))) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k_col<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem_col_bytes<T>(maxN))) != cudaSuccess)
        return e;
    return cudaFuncSetAttribute(k_row_inv<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem_row_inv_bytes<T>(maxN));
}

template <typename T>
cudaError_t launch_row_fwd(const SolveArgs<T> &a, int n_items, cudaStream_t st)
{
    k_row_fwd<T><<<n_items, fft_threads(a.N, 2), smem_row_fwd_bytes<T>(a.N), st>>>(a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_col(const SolveArgs<T> &a, int n_outputs, cudaStream_t st)
{
    dim3 grid(a.N + 1, n_outputs);
    k_col<T><<<grid, fft_threads(a.N, 2), smem_col_bytes<T>(a.N), st>>>(a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_row_inv(const SolveArgs<T> &a, cudaStream_t st)
{
    dim3 grid(a.N / 2, a.L);
    k_row_inv<T><<<grid, fft_threads(a.N, 2), smem_row_inv_bytes<T>(a.N), st>>>(a);
    return cudaGetLastError();
}

template cudaError_t launch_restrict<float>(const float *, float *, const float *, int, int, int, cudaStream_t);
template cudaError_t launch_restrict<double>(const double *, double *, const double *, int, int, int, cudaStream_t);
template cudaError_t launch_row_fwd<float>(const SolveArgs<float> &, int, cudaStream_t);
template cudaError_t launch_row_fwd<double>(const SolveArgs<double> &, int, cudaStream_t);
template cudaError_t launch_col<float>(const SolveArgs<float> &, int, cudaStream_t);
template cudaError_t launch_col<double>(const SolveArgs<double> &, int, cudaStream_t);
template cudaError_t launch_row_inv<float>(const SolveArgs<float> &, cudaStream_t);
template cudaError_t launch_row_inv<double>(const SolveArgs<double> &, cudaStream_t);
template size_t smem_col_bytes<float>(int);
template size_t smem_col_bytes<double>(int);
template cudaError_t solve_kernels_init<float>();
template cudaError_t solve_kernels_init<double>();

}  // namespace sgf
