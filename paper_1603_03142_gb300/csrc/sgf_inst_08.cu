// sgf_inst_08.cu -- transform-pass instances for N = 256.
#include "sgf_kernels.cuh"

namespace sgf {
template cudaError_t launch_pass<float, 8>(int, const SolveArgs<float> &, int, cudaStream_t, const BatchView<float> *);
template cudaError_t launch_pass<double, 8>(int, const SolveArgs<double> &, int, cudaStream_t, const BatchView<double> *);
}  // namespace sgf
