// sgf_inst_12.cu -- transform-pass instances for N = 4096 (FP32 and FP64 paths).
#include "sgf_kernels.cuh"

namespace sgf {
template cudaError_t launch_pass<float, 12, false>(int, const SolveArgs<float> &, int, cudaStream_t, const BatchView<float> *);
}  // namespace sgf
