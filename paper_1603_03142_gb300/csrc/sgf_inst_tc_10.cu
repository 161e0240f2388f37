// sgf_inst_tc_10.cu -- transform-pass instances for N = 1024, SGF_BF16X (tensor-core tiles).
#include "sgf_kernels.cuh"

namespace sgf {
template cudaError_t launch_pass<float, 10, true>(int, const SolveArgs<float> &, int, cudaStream_t, const BatchView<float> *);
}  // namespace sgf
