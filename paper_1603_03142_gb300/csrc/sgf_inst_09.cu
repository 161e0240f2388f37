// sgf_inst_09.cu -- transform-pass instances for N = 512.
#include "sgf_kernels.cuh"

namespace sgf {
template cudaError_t launch_pass<float, 9>(int, const SolveArgs<float> &, int, cudaStream_t, const BatchView<float> *);
template cudaError_t launch_pass<double, 9>(int, const SolveArgs<double> &, int, cudaStream_t, const BatchView<double> *);
}  // namespace sgf
