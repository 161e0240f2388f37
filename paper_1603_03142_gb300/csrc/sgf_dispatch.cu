// sgf_dispatch.cu -- selects the compile-time instance of a transform pass
// for the plan's N (instances live in sgf_inst_<logN>.cu) and precision path.
#include "sgf_kernels.cuh"

namespace sgf {

#define SGF_EXTERN(T, LOGN, TC) \
    extern template cudaError_t launch_pass<T, LOGN, TC>(int, const SolveArgs<T> &, int, cudaStream_t, const BatchView<T> *);
SGF_EXTERN(double, 4, false)
SGF_EXTERN(float, 4, false)
SGF_EXTERN(float, 4, true)
SGF_EXTERN(double, 5, false)
SGF_EXTERN(float, 5, false)
SGF_EXTERN(float, 5, true)
SGF_EXTERN(double, 6, false)
SGF_EXTERN(float, 6, false)
SGF_EXTERN(float, 6, true)
SGF_EXTERN(double, 7, false)
SGF_EXTERN(float, 7, false)
SGF_EXTERN(float, 7, true)
SGF_EXTERN(double, 8, false)
SGF_EXTERN(float, 8, false)
SGF_EXTERN(float, 8, true)
SGF_EXTERN(double, 9, false)
SGF_EXTERN(float, 9, false)
SGF_EXTERN(float, 9, true)
SGF_EXTERN(double, 10, false)
SGF_EXTERN(float, 10, false)
SGF_EXTERN(float, 10, true)
SGF_EXTERN(double, 11, false)
SGF_EXTERN(float, 11, false)
SGF_EXTERN(float, 11, true)
SGF_EXTERN(float, 12, false)
SGF_EXTERN(float, 12, true)
#undef SGF_EXTERN

template <typename T>
cudaError_t launch_pass_n(int pass, int logN, const SolveArgs<T> &a, int count, cudaStream_t st,
                          const BatchView<T> *bv, bool tc)
{
    if constexpr (sizeof(T) == 4) {
        if (tc) {
            switch (logN) {
            case 4: return launch_pass<T, 4, true>(pass, a, count, st, bv);
            case 5: return launch_pass<T, 5, true>(pass, a, count, st, bv);
            case 6: return launch_pass<T, 6, true>(pass, a, count, st, bv);
            case 7: return launch_pass<T, 7, true>(pass, a, count, st, bv);
            case 8: return launch_pass<T, 8, true>(pass, a, count, st, bv);
            case 9: return launch_pass<T, 9, true>(pass, a, count, st, bv);
            case 10: return launch_pass<T, 10, true>(pass, a, count, st, bv);
            case 11: return launch_pass<T, 11, true>(pass, a, count, st, bv);
            case 12: return launch_pass<T, 12, true>(pass, a, count, st, bv);
            default: return cudaErrorInvalidValue;
            }
        }
    } else if (tc) {
        return cudaErrorInvalidValue;
    }
    switch (logN) {
    case 4: return launch_pass<T, 4, false>(pass, a, count, st, bv);
    case 5: return launch_pass<T, 5, false>(pass, a, count, st, bv);
    case 6: return launch_pass<T, 6, false>(pass, a, count, st, bv);
    case 7: return launch_pass<T, 7, false>(pass, a, count, st, bv);
    case 8: return launch_pass<T, 8, false>(pass, a, count, st, bv);
    case 9: return launch_pass<T, 9, false>(pass, a, count, st, bv);
    case 10: return launch_pass<T, 10, false>(pass, a, count, st, bv);
    case 11: return launch_pass<T, 11, false>(pass, a, count, st, bv);
    case 12:
        if constexpr (sizeof(T) == 4)
            return launch_pass<T, 12, false>(pass, a, count, st, bv);
        else
            return cudaErrorInvalidValue;
    default:
        return cudaErrorInvalidValue;
    }
}

template cudaError_t launch_pass_n<float>(int, int, const SolveArgs<float> &, int, cudaStream_t,
                                         const BatchView<float> *, bool);
template cudaError_t launch_pass_n<double>(int, int, const SolveArgs<double> &, int, cudaStream_t,
                                          const BatchView<double> *, bool);

}  // namespace sgf
