// sgf_dispatch.cu -- selects the compile-time instance of a transform pass
// for the plan's N (instances live in sgf_inst_<logN>.cu).
#include "sgf_kernels.cuh"

namespace sgf {

extern template cudaError_t launch_pass<float, 4>(int, const SolveArgs<float> &, int, cudaStream_t, const BatchView<float> *);
extern template cudaError_t launch_pass<double, 4>(int, const SolveArgs<double> &, int, cudaStream_t, const BatchView<double> *);
extern template cudaError_t launch_pass<float, 5>(int, const SolveArgs<float> &, int, cudaStream_t, const BatchView<float> *);
extern template cudaError_t launch_pass<double, 5>(int, const SolveArgs<double> &, int, cudaStream_t, const BatchView<double> *);
extern template cudaError_t launch_pass<float, 6>(int, const SolveArgs<float> &, int, cudaStream_t, const BatchView<float> *);
extern template cudaError_t launch_pass<double, 6>(int, const SolveArgs<double> &, int, cudaStream_t, const BatchView<double> *);
extern template cudaError_t launch_pass<float, 7>(int, const SolveArgs<float> &, int, cudaStream_t, const BatchView<float> *);
extern template cudaError_t launch_pass<double, 7>(int, const SolveArgs<double> &, int, cudaStream_t, const BatchView<double> *);
extern template cudaError_t launch_pass<float, 8>(int, const SolveArgs<float> &, int, cudaStream_t, const BatchView<float> *);
extern template cudaError_t launch_pass<double, 8>(int, const SolveArgs<double> &, int, cudaStream_t, const BatchView<double> *);
extern template cudaError_t launch_pass<float, 9>(int, const SolveArgs<float> &, int, cudaStream_t, const BatchView<float> *);
extern template cudaError_t launch_pass<double, 9>(int, const SolveArgs<double> &, int, cudaStream_t, const BatchView<double> *);
extern template cudaError_t launch_pass<float, 10>(int, const SolveArgs<float> &, int, cudaStream_t, const BatchView<float> *);
extern template cudaError_t launch_pass<double, 10>(int, const SolveArgs<double> &, int, cudaStream_t, const BatchView<double> *);
extern template cudaError_t launch_pass<float, 11>(int, const SolveArgs<float> &, int, cudaStream_t, const BatchView<float> *);
extern template cudaError_t launch_pass<double, 11>(int, const SolveArgs<double> &, int, cudaStream_t, const BatchView<double> *);
extern template cudaError_t launch_pass<float, 12>(int, const SolveArgs<float> &, int, cudaStream_t, const BatchView<float> *);

template <typename T>
cudaError_t launch_pass_n(int pass, int logN, const SolveArgs<T> &a, int count, cudaStream_t st,
                          const BatchView<T> *bv)
{
    switch (logN) {
    case 4: return launch_pass<T, 4>(pass, a, count, st, bv);
    case 5: return launch_pass<T, 5>(pass, a, count, st, bv);
    case 6: return launch_pass<T, 6>(pass, a, count, st, bv);
    case 7: return launch_pass<T, 7>(pass, a, count, st, bv);
    case 8: return launch_pass<T, 8>(pass, a, count, st, bv);
    case 9: return launch_pass<T, 9>(pass, a, count, st, bv);
    case 10: return launch_pass<T, 10>(pass, a, count, st, bv);
    case 11: return launch_pass<T, 11>(pass, a, count, st, bv);
    case 12:
        if constexpr (sizeof(T) == 4)
            return launch_pass<T, 12>(pass, a, count, st, bv);
        else
            return cudaErrorInvalidValue;
    default:
        return cudaErrorInvalidValue;
    }
}

template cudaError_t launch_pass_n<float>(int, int, const SolveArgs<float> &, int, cudaStream_t,
                                         const BatchView<float> *);
template cudaError_t launch_pass_n<double>(int, int, const SolveArgs<double> &, int, cudaStream_t,
                                          const BatchView<double> *);

}  // namespace sgf
