// sgf_host.h -- host-side helpers shared by the translation units of the C ABI.
#pragma once
#include <cuda_runtime.h>
#include <string>

#include "../../include/sgf.h"

namespace sgf {
// Records a printf-style message as the calling thread's last error (sgf_last_error)
// and returns s.
sgf_status fail(sgf_status s, const char *fmt, ...);
// fail() for a CUDA runtime error: SGF_ENOMEM for an allocation failure, SGF_ECUDA otherwise.
sgf_status cuda_fail(cudaError_t e, const char *what);
}  // namespace sgf
