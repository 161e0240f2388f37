// sgf_inst_06.cu -- transform-pass instances for N = 64 (FP32 and FP64 paths).
#include "sgf_kernels.cuh"

namespace sgf {
template cudaError_t launch_pass<float, 6, false>(int, const SolveArgs<float> &, int, cudaStream_t, const BatchView<float> *);
template cudaError_t launch_pass<double, 6, false>(int, const SolveArgs<double> &, int, cudaStream_t, const BatchView<double> *);
}  // namespace sgf
