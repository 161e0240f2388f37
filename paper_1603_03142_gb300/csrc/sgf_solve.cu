// sgf_solve.cu -- restriction kernel of libsgf.
//
// Every covered cell of level l takes the mean of its four children on level
// l+1 (recursively from the finest level).  These values only feed the slopes
// of the uncovered neighbours (Sec. 2.1 slope reading); covered cells carry no
// mass.  The transform kernels are in sgf_solve16.cu.
#include "sgf_internal.h"

namespace sgf {

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

template <typename T>
__global__ void k_restrict_batch(const SolveArgs<T> *__restrict__ args, const int2 *__restrict__ jobs)
{
    const int2 job = jobs[blockIdx.y];
    const SolveArgs<T> &a = args[job.x];
    const int l = job.y, N = a.N;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= N * N)
        return;
    const int j = idx / N, i = idx - j * N;
    const int half = N >> 1, ox = a.child_ox[l], oy = a.child_oy[l];
    T v = a.sigma_in[l][idx];
    if (i >= ox && i < ox + half && j >= oy && j < oy + half) {
        const T *f = a.src[l + 1] + (size_t)(2 * (j - oy)) * N + 2 * (i - ox);
        v = T(0.25) * ((f[0] + f[1]) + (f[N] + f[N + 1]));
    }
    const_cast<T *>(a.src[l])[idx] = v;
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

template cudaError_t launch_restrict<float>(const float *, float *, const float *, int, int, int, cudaStream_t);
template cudaError_t launch_restrict<double>(const double *, double *, const double *, int, int, int, cudaStream_t);

}  // namespace sgf
