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

template cudaError_t launch_restrict_batch<float>(const SolveArgs<float> *, const int2 *, int, int, cudaStream_t);
template cudaError_t launch_restrict_batch<double>(const SolveArgs<double> *, const int2 *, int, int, cudaStream_t);

template cudaError_t launch_restrict<float>(const SolveArgs<float> &, int, cudaStream_t);
template cudaError_t launch_restrict<double>(const SolveArgs<double> &, int, cudaStream_t);

}  // namespace sgf
