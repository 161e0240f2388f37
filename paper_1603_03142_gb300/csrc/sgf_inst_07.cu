// sgf_inst_07.cu -- transform-pass instances for N = 128 (FP32 and FP64 paths).
#include "sgf_kernels.cuh"

namespace sgf {
template cudaError_t launch_pass<float, 7, false>(int, const SolveArgs<float> &, int, cudaStream_t, const BatchView<float> *);
template cudaError_t launch_pass<double, 7, false>(int, const SolveArgs<double> &, int, cudaStream_t, const BatchView<double> *);
}  // namespace sgf
