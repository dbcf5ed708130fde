// Serve-loop kernels for f32 rows (one translation unit per format, so the
// formats compile in parallel).
#include "serve_launch.cuh"

namespace jag {
template cudaError_t launch_serve_fmt<JAG_VEC_F32>(const ServeArgs &, int, cudaStream_t, int *);
}  // namespace jag
