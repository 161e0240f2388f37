// sgf_inst_10.cu -- transform-pass instances for N = 1024 (FP32 and FP64 paths).
#include "sgf_kernels.cuh"

namespace sgf {
template cudaError_t launch_pass<float, 10, false>(int, const SolveArgs<float> &, int, cudaStream_t, const BatchView<float> *);
template cudaError_t launch_pass<double, 10, false>(int, const SolveArgs<double> &, int, cudaStream_t, const BatchView<double> *);
}  // namespace sgf
