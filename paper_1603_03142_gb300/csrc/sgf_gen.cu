// sgf_gen.cu -- FP64 kernel tables and their spectra (plan time).
//
// For one pair of levels (and one phase of it), every table entry is the exact
// integral over one source cell of the force kernel times the linear density
// of Eq. (eqnSigma), for a target at the origin, in units of the finer of the
// two cell sizes.  Writing u = xb - x_t, v = yb - y_t, r = |(u, v)| and
// DD[g] = g(b,d) - g(a,d) - g(b,c) + g(a,c) over the cell [a,b] x [c,d]:
//   Int u/r^3   = DD[-ln(v + r)]   (Eq. eqnCalK; the (0, v) branch is -sgn(v) ln|v|)
//   Int v/r^3   = the same with u and v exchanged
//   Int u^2/r^3 = DD[v ln(u + r)]
//   Int v^2/r^3 = DD[u ln(v + r)]
//   Int uv/r^3  = DD[-r]
// Terms of an antiderivative that depend on only one of u, v cancel in DD
// exactly, so the device evaluates  -ln(v + r) = -asinh(v/|u|) - ln|u|  as
// -asinh(v/|u|), and  v ln(u + r)  as  v asinh(u/|v|);  asinh keeps every
// digit where v + r would cancel (v < 0).  At a corner with u = v = 0 (only
// reachable by targets under a finer patch, whose output is zeroed) every
// antiderivative is taken as 0, so no table entry is ever NaN.
//
// Tables (lattice units, slope kernels expanded about the source centre
// (u_c, v_c), Sec. 2.1):
//   K0x = Int u/r^3,  Kxx = Int u^2/r^3 - u_c K0x,  Kxy = Int uv/r^3 - v_c K0x,
//   K0y = Int v/r^3,  Kyx = Int uv/r^3 - u_c K0y,   Kyy = Int v^2/r^3 - v_c K0y.
// The solve feeds per-cell differences (slope x source cell size), so the
// slope tables are scaled by (finer cell)/(source cell): 1/m in Case 3.
//
// Index d of a table is the convolution index of Sec. 2.1 (target minus
// source, in the phase lattice), stored at d mod P.  Per axis the source
// cell's lower edge and width, in units of the finer cell, are
//   Case 1: lo = -d - 1/2,              w = 1,  d in [-(N-1), N-1]
//   Case 2: lo = -m d + p - m/2 + A,    w = 1,  d in [-(N/m-1), N-1]   (p: source phase,
//                                                A: source corner minus target corner)
//   Case 3: lo = -m d - p - A - 1/2,    w = m,  d in [-(N-1), N/m-1]   (p: target phase,
//                                                A: target corner minus source corner)
// and each set is transformed in FP64 (P x P, P = 2N) and scaled by 1/P^2.
//
// Potential sets (kernel -1/r, Sec. 2): with the same DD and conventions
//   Int 1/r = DD[u ln(v + r) + v ln(u + r)]
//   Int u/r = DD[(v r + u^2 ln(v + r)) / 2]
//   Int v/r = DD[(u r + v^2 ln(u + r)) / 2]
// (one-variable terms dropped as above: u ln(v + r) -> u asinh(v/|u|)), and
//   P0 = -h Int 1/r,  Px = -h (Int u/r - u_c Int 1/r),  Py = -h (Int v/r - v_c Int 1/r),
// h the finer cell size of the pair (the force tables are scale-free, the
// potential grows with the cell), the slope tables again scaled by 1/m in Case 3.
#include "sgf_fft.cuh"
#include "sgf_internal.h"

namespace sgf {

struct Corner {
    double g0x, g0y, hxx, hyy, hxy;
};

__device__ __forceinline__ Corner corner_eval(double u, double v)
{
    Corner k;
    const double au = fabs(u), av = fabs(v);
    const double A = au > 0.0 ? asinh(v / au) : 0.0;  // asinh(v/|u|)
    const double B = av > 0.0 ? asinh(u / av) : 0.0;  // asinh(u/|v|)
    if (au > 0.0)
        k.g0x = -A;
    else
        k.g0x = av > 0.0 ? -copysign(log(av), v) : 0.0;
    if (av > 0.0)
        k.g0y = -B;
    else
        k.g0y = au > 0.0 ? -copysign(log(au), u) : 0.0;
    k.hxx = av > 0.0 ? v * B : 0.0;
    k.hyy = au > 0.0 ? u * A : 0.0;
    k.hxy = -hypot(u, v);
    return k;
}

// Corner values of the potential antiderivatives: (Int 1/r, Int u/r, Int v/r).
__device__ __forceinline__ void corner_phi(double u, double v, double k[3])
{
    const double au = fabs(u), av = fabs(v);
    const double r = hypot(u, v);
    const double lu = au > 0.0 ? u * asinh(v / au) : 0.0;  // u ln(v + r), less u ln|u|
    const double lv = av > 0.0 ? v * asinh(u / av) : 0.0;  // v ln(u + r), less v ln|v|
    k[0] = lu + lv;
    k[1] = 0.5 * (v * r + u * lu);
    k[2] = 0.5 * (u * r + v * lv);
}

struct AxisMap {
    int cas, m, p, A, N;
    __device__ __forceinline__ bool index(int pos, int P, int &d) const
    {
        int dmin, dmax;
        if (cas == 1) { dmin = -(N - 1); dmax = N - 1; }
        else if (cas == 2) { dmin = -(N / m - 1); dmax = N - 1; }
        else { dmin = -(N - 1); dmax = N / m - 1; }
        if (pos <= dmax) { d = pos; return true; }
        if (pos - P >= dmin) { d = pos - P; return true; }
        return false;
    }
    __device__ __forceinline__ void edges(int d, double &lo, double &w) const
    {
        if (cas == 1) { lo = -d - 0.5; w = 1.0; }
        else if (cas == 2) { lo = -(double)m * d + p - 0.5 * m + A; w = 1.0; }
        else { lo = -(double)m * d - p - A - 0.5; w = (double)m; }
    }
};

// The six tables of one source cell at convolution index (dx, dy).
__device__ __forceinline__ void cell_tables(const AxisMap &mx, const AxisMap &my, int dx, int dy, int cas, int m,
                                            double out[6])
{
    double a, wx, c, wy;
    mx.edges(dx, a, wx);
    my.edges(dy, c, wy);
    const double b = a + wx, d = c + wy;
    const Corner k1 = corner_eval(b, d), k2 = corner_eval(a, d), k3 = corner_eval(b, c), k4 = corner_eval(a, c);
    const double i0x = (k1.g0x - k2.g0x) - (k3.g0x - k4.g0x);
    const double i0y = (k1.g0y - k3.g0y) - (k2.g0y - k4.g0y);
    const double ixx = (k1.hxx - k2.hxx) - (k3.hxx - k4.hxx);
    const double iyy = (k1.hyy - k3.hyy) - (k2.hyy - k4.hyy);
    const double ixy = (k1.hxy - k2.hxy) - (k3.hxy - k4.hxy);
    const double uc = a + 0.5 * wx, vc = c + 0.5 * wy;
    const double sf = cas == 3 ? 1.0 / m : 1.0;
    out[0] = i0x;
    out[1] = (ixx - uc * i0x) * sf;
    out[2] = (ixy - vc * i0x) * sf;
    out[3] = i0y;
    out[4] = (ixy - uc * i0y) * sf;
    out[5] = (iyy - vc * i0y) * sf;
}

// The three potential tables of one source cell at convolution index (dx, dy).
__device__ __forceinline__ void cell_tables_phi(const AxisMap &mx, const AxisMap &my, int dx, int dy, int cas, int m,
                                                double h, double out[3])
{
    double a, wx, c, wy;
    mx.edges(dx, a, wx);
    my.edges(dy, c, wy);
    const double b = a + wx, d = c + wy;
    double k1[3], k2[3], k3[3], k4[3];
    corner_phi(b, d, k1);
    corner_phi(a, d, k2);
    corner_phi(b, c, k3);
    corner_phi(a, c, k4);
    double I[3];
    for (int q = 0; q < 3; ++q)
        I[q] = (k1[q] - k2[q]) - (k3[q] - k4[q]);
    const double uc = a + 0.5 * wx, vc = c + 0.5 * wy;
    const double sf = cas == 3 ? 1.0 / m : 1.0;
    out[0] = -h * I[0];
    out[1] = -h * sf * (I[1] - uc * I[0]);
    out[2] = -h * sf * (I[2] - vc * I[0]);
}

// Case 1 with the central-difference slope stencils folded in (zero-rim
// single level): dx = (s[i+1] - s[i-1])/2 gives
//   sum_s Kxx[t-s] dx[s] = sum_s s[s] (Kxx[d + x] - Kxx[d - x])/2,  d = t - s,
// so Gx = K0x + (Kxx[d+x] - Kxx[d-x])/2 + (Kxy[d+y] - Kxy[d-y])/2 and
//    Gy = K0y + (Kyx[d+x] - Kyx[d-x])/2 + (Kyy[d+y] - Kyy[d-y])/2,
// with the neighbouring entries evaluated exactly (they may lie one cell
// beyond the table's range).
__device__ __forceinline__ void merged_tables(const AxisMap &mx, const AxisMap &my, int dx, int dy, double out[2])
{
    double c0[6], xp[6], xm[6], yp[6], ym[6];
    cell_tables(mx, my, dx, dy, 1, 1, c0);
    cell_tables(mx, my, dx + 1, dy, 1, 1, xp);
    cell_tables(mx, my, dx - 1, dy, 1, 1, xm);
    cell_tables(mx, my, dx, dy + 1, 1, 1, yp);
    cell_tables(mx, my, dx, dy - 1, 1, 1, ym);
    out[0] = c0[0] + 0.5 * (xp[1] - xm[1]) + 0.5 * (yp[2] - ym[2]);
    out[1] = c0[3] + 0.5 * (xp[4] - xm[4]) + 0.5 * (yp[5] - ym[5]);
}

// The potential's zero-rim table: P0 + (Px[d + x] - Px[d - x])/2 + (Py[d + y] - Py[d - y])/2
// (the same stencil algebra as merged_tables).
__device__ __forceinline__ void merged_tables_phi(const AxisMap &mx, const AxisMap &my, int dx, int dy, double h,
                                                  double out[1])
{
    double c0[3], xp[3], xm[3], yp[3], ym[3];
    cell_tables_phi(mx, my, dx, dy, 1, 1, h, c0);
    cell_tables_phi(mx, my, dx + 1, dy, 1, 1, h, xp);
    cell_tables_phi(mx, my, dx - 1, dy, 1, 1, h, xm);
    cell_tables_phi(mx, my, dx, dy + 1, 1, 1, h, yp);
    cell_tables_phi(mx, my, dx, dy - 1, 1, 1, h, ym);
    out[0] = c0[0] + 0.5 * (xp[1] - xm[1]) + 0.5 * (yp[2] - ym[2]);
}

__global__ void k_gen_tables(GenSet g, int N, double *__restrict__ tables)
{
    const int P = 2 * N;
    const int px = blockIdx.x * blockDim.x + threadIdx.x;
    const int py = blockIdx.y;
    if (px >= P)
        return;
    const int cas = g.cas == 4 ? 1 : g.cas;
    const AxisMap mx{cas, g.m, g.px, g.ax, N}, my{cas, g.m, g.py, g.ay, N};
    double out[6] = {0, 0, 0, 0, 0, 0};
    int dx, dy;
    const int ntab = spec_tables(g.kind);
    if (mx.index(px, P, dx) && my.index(py, P, dy)) {
        if (g.kind == SPEC_MERGED_PHI)
            merged_tables_phi(mx, my, dx, dy, g.h, out);
        else if (g.cas == 4)
            merged_tables(mx, my, dx, dy, out);
        else if (spec_phi(g.kind))
            cell_tables_phi(mx, my, dx, dy, g.cas, g.m, g.h, out);
        else
            cell_tables(mx, my, dx, dy, g.cas, g.m, out);
    }
    const size_t plane = (size_t)P * P, at = (size_t)py * P + px;
    for (int t = 0; t < ntab; ++t)
        tables[t * plane + at] = out[t];
}

// Rows of the P x P tables -> half spectra along x: half[t][kx 0..N][y 0..P).
// Two real rows ride as one complex row; the P-point transform of a row is
// folded into two N-point transforms: bin 2k+b = DFT_N[(x[n] + (-1)^b x[n+N]) W_P^{bn}].
__global__ void k_gen_rows(int N, int logN, const double *__restrict__ tables,
                           double2 *__restrict__ half, const double2 *__restrict__ tw)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2 *W = reinterpret_cast<double2 *>(smem_raw);
    const int P = 2 * N, tid = threadIdx.x, nt = blockDim.x;
    const int t = blockIdx.y, y0 = 2 * blockIdx.x;
    const double *ra = tables + (size_t)t * P * P + (size_t)y0 * P;
    const double *rb = ra + P;
    for (int n = tid; n < N; n += nt) {
        const double2 lo = make_double2(ra[n], rb[n]), hi = make_double2(ra[n + N], rb[n + N]);
        W[n] = make_double2(lo.x + hi.x, lo.y + hi.y);
        W[N + n] = cmul(make_double2(lo.x - hi.x, lo.y - hi.y), tw[n]);
    }
    __syncthreads();
    block_fft<double2, false>(W, N, logN, 2, tw);
    double2 *out = half + (size_t)t * (N + 1) * P;
    for (int kx = tid; kx <= N; kx += nt) {
        const int b = kx & 1, k = kx >> 1;
        const int km = (N - b - k) & (N - 1);
        const double2 Z = W[b * N + k], Zm = cconj(W[b * N + km]);
        const double2 s = cadd(Z, Zm), d = csub(Z, Zm);
        out[(size_t)kx * P + y0] = make_double2(0.5 * s.x, 0.5 * s.y);
        out[(size_t)kx * P + y0 + 1] = make_double2(0.5 * d.y, -0.5 * d.x);
    }
}

// Columns kx of the half spectra -> the stored kernel spectra (scaled by 1/P^2).
template <typename T>
__global__ void k_gen_cols(int N, int logN, const double2 *__restrict__ half, const double2 *__restrict__ tw,
                           int kind, void *spec, size_t spec_off)
{
    using C = typename std::conditional<sizeof(T) == 8, double2, float2>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2 *W = reinterpret_cast<double2 *>(smem_raw);
    const int P = 2 * N, tid = threadIdx.x, nt = blockDim.x;
    const int kx = blockIdx.x, t = blockIdx.y;
    const double2 *col = half + ((size_t)t * (N + 1) + kx) * P;
    for (int n = tid; n < N; n += nt) {
        const double2 lo = col[n], hi = col[n + N];
        W[n] = cadd(lo, hi);
        W[N + n] = cmul(csub(lo, hi), tw[n]);
    }
    __syncthreads();
    block_fft<double2, false>(W, N, logN, 2, tw);
    const double scale = 1.0 / ((double)P * (double)P);
    if (spec_quarter(kind) || kind == SPEC_MERGED || kind == SPEC_MERGED_PHI) {
        // K0x and K0y (tables 0, 3) are odd in one axis: purely imaginary; merged Gx, Gy
        // too; of the potential tables Px and Py (1, 2), while P0 is real
        const int QS = quarter_stride(N), HQ = quarter_half(N);
        T *dst = reinterpret_cast<T *>(spec) + spec_off + ((size_t)t * (N + 1) + kx) * QS;
        const bool imag = kind == SPEC_MERGED ||
                          (kind == SPEC_MERGED_PHI ? false : kind == SPEC_QUARTER_PHI ? t != 0 : t == 0 || t == 3);
        for (int idx = tid; idx < QS; idx += nt) {
            const int q = idx < HQ ? 2 * idx : 2 * (idx - HQ) + 1;  // even half, then odd half
            const double2 X = q <= N ? W[(q & 1) * N + (q >> 1)] : make_double2(0.0, 0.0);
            dst[idx] = (T)((imag ? X.y : X.x) * scale);
        }
    } else {
        C *dst = reinterpret_cast<C *>(spec) + spec_off + ((size_t)t * (N + 1) + kx) * P;
        for (int ky = tid; ky < P; ky += nt) {
            const double2 X = W[(ky & 1) * N + (ky >> 1)];
            C v;
            v.x = (T)(X.x * scale);
            v.y = (T)(X.y * scale);
            dst[ky] = v;
        }
    }
}

static inline int gen_threads(int N)
{
    int nt = (2 * N) / kFftVpt;
    if (nt < 64)
        nt = 64;
    if (nt > 1024)
        nt = 1024;
    return nt;
}

cudaError_t gen_kernels_init()
{
    const int bytes = (int)(2 * 4096 * sizeof(double2));
    cudaError_t e = cudaFuncSetAttribute(k_gen_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess)
        return e;
    e = cudaFuncSetAttribute(k_gen_cols<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess)
        return e;
    return cudaFuncSetAttribute(k_gen_cols<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

template <typename T>
cudaError_t launch_gen_set(const GenSet &g, int N, int logN, const double2 *tw64, void *spec,
                           double *work_tables, double2 *work_half, cudaStream_t st)
{
    const int P = 2 * N;
    {
        const int bs = 256;
        dim3 grid((P + bs - 1) / bs, P);
        k_gen_tables<<<grid, bs, 0, st>>>(g, N, work_tables);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    const size_t smem = 2 * (size_t)N * sizeof(double2);
    const int ntab = spec_tables(g.kind);
    k_gen_rows<<<dim3(P / 2, ntab), gen_threads(N), smem, st>>>(N, logN, work_tables, work_half, tw64);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return e;
    k_gen_cols<T><<<dim3(N + 1, ntab), gen_threads(N), smem, st>>>(N, logN, work_half, tw64, g.kind, spec,
                                                                     g.spec_off);
    return cudaGetLastError();
}

template cudaError_t launch_gen_set<float>(const GenSet &, int, int, const double2 *, void *, double *,
                                           double2 *, cudaStream_t);
template cudaError_t launch_gen_set<double>(const GenSet &, int, int, const double2 *, void *, double *,
                                            double2 *, cudaStream_t);

}  // namespace sgf
