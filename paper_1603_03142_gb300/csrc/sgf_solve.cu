// sgf_solve.cu -- restriction kernel of libsgf.
//
// Every covered cell of a patch takes the mean of its four children on the
// finer patch over it (finest patches first, so the children are restricted
// values themselves where they are covered in turn).  These values only feed
// the slopes of the uncovered neighbours (Sec. 2.1 slope reading); covered
// cells carry no mass.  The transform kernels are in sgf_kernels.cuh.
#include "sgf_internal.h"

namespace sgf {

// ------------------------------------------------------------------ restrict
template <typename T>
__device__ __forceinline__ void restrict_cell(const SolveArgs<T> &a, int p, int idx)
{
    const int N = a.N;
    const int j = idx / N, i = idx - j * N;
    T v = a.sigma_in[p][idx];
    for (int k = a.cover_begin[p]; k < a.cover_begin[p + 1]; ++k) {
        const CoverRect &r = a.cover[k];
        if (i >= r.x0 && i < r.x1 && j >= r.y0 && j < r.y1) {
            const T *f = a.src[r.fine] + (size_t)(2 * (j - r.fy)) * N + 2 * (i - r.fx);
            v = T(0.25) * ((f[0] + f[1]) + (f[N] + f[N + 1]));
            break;
        }
    }
    const_cast<T *>(a.src[p])[idx] = v;
}

template <typename T>
__global__ void k_restrict(SolveArgs<T> a, int p)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < a.N * a.N)
        restrict_cell(a, p, idx);
}

template <typename T>
cudaError_t launch_restrict(const SolveArgs<T> &a, int p, cudaStream_t st)
{
    const int n = a.N * a.N, bs = 256;
    k_restrict<T><<<(n + bs - 1) / bs, bs, 0, st>>>(a, p);
    return cudaGetLastError();
}

template <typename T>
__global__ void k_restrict_batch(const SolveArgs<T> *__restrict__ args, const int2 *__restrict__ jobs)
{
    const int2 job = jobs[blockIdx.y];
    const SolveArgs<T> &a = args[job.x];
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < a.N * a.N)
        restrict_cell(a, job.y, idx);
}

template <typename T>
cudaError_t launch_restrict_batch(const SolveArgs<T> *args, const int2 *jobs, int njobs, int max_n, cudaStream_t st)
{
    if (njobs <= 0)
        return cudaSuccess;
    const int bs = 256;
    dim3 grid((max_n * max_n + bs - 1) / bs, njobs);
    k_restrict_batch<T><<<grid, bs, 0, st>>>(args, jobs);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- embedding
// A plan whose patches have n cells a side below its transform size N solves
// them embedded in N x N arrays: the densities are copied in with zeros beyond
// n, the forces copied back.
template <typename T>
__global__ void k_pad(IoPtrs<T> io, int n, int N)
{
    const int l = blockIdx.y;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= N * N)
        return;
    const int j = idx / N, i = idx - j * N;
    io.dst[l][idx] = i < n && j < n ? io.src[l][(size_t)j * n + i] : T(0);
}

template <typename T>
__global__ void k_crop(IoPtrs<T> io, int n, int N)
{
    const int l = blockIdx.y;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * n)
        return;
    const int j = idx / n, i = idx - j * n;
    io.dst[l][idx] = io.src[l][(size_t)j * N + i];
}

template <typename T>
cudaError_t launch_pad(const IoPtrs<T> &io, int L, int n, int N, cudaStream_t st)
{
    const int bs = 256;
    k_pad<T><<<dim3((N * N + bs - 1) / bs, L), bs, 0, st>>>(io, n, N);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_crop(const IoPtrs<T> &io, int L, int n, int N, cudaStream_t st)
{
    const int bs = 256;
    k_crop<T><<<dim3((n * n + bs - 1) / bs, L), bs, 0, st>>>(io, n, N);
    return cudaGetLastError();
}

template cudaError_t launch_pad<float>(const IoPtrs<float> &, int, int, int, cudaStream_t);
template cudaError_t launch_pad<double>(const IoPtrs<double> &, int, int, int, cudaStream_t);
template cudaError_t launch_crop<float>(const IoPtrs<float> &, int, int, int, cudaStream_t);
template cudaError_t launch_crop<double>(const IoPtrs<double> &, int, int, int, cudaStream_t);

template cudaError_t launch_restrict_batch<float>(const SolveArgs<float> *, const int2 *, int, int, cudaStream_t);
template cudaError_t launch_restrict_batch<double>(const SolveArgs<double> *, const int2 *, int, int, cudaStream_t);

template cudaError_t launch_restrict<float>(const SolveArgs<float> &, int, cudaStream_t);
template cudaError_t launch_restrict<double>(const SolveArgs<double> &, int, cudaStream_t);

}  // namespace sgf
