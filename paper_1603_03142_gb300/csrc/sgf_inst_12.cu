// sgf_inst_12.cu -- transform-pass instances for N = 4096.
#include "sgf_kernels.cuh"

namespace sgf {
template cudaError_t launch_pass<float, 12>(int, const SolveArgs<float> &, int, cudaStream_t, const BatchView<float> *);
}  // namespace sgf
