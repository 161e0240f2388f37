// sgf_inst_07.cu -- transform-pass instances for N = 128.
#include "sgf_kernels.cuh"

namespace sgf {
template cudaError_t launch_pass<float, 7>(int, const SolveArgs<float> &, int, cudaStream_t, const BatchView<float> *);
template cudaError_t launch_pass<double, 7>(int, const SolveArgs<double> &, int, cudaStream_t, const BatchView<double> *);
}  // namespace sgf
