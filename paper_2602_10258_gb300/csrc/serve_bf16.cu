// Serve-loop kernels for bf16 rows (one translation unit per format, so the
// formats compile in parallel).
#include "serve_launch.cuh"

namespace jag {
template cudaError_t launch_serve_fmt<JAG_VEC_BF16>(const ServeArgs &, int, cudaStream_t, int *);
}  // namespace jag
