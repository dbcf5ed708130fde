// K4: BF16 / FP8-E4M3 rows of an index from its fp32 rows.
//   BF16: each element rounded to nearest (ties to even), scale 1.
//   FP8:  per-row scale s = max|x_i| / 448 (1 for a zero row); each element
//         x_i / s rounded to the nearest E4M3 value (ties to even),
//         saturating at +-448.
// Rows are zero padded to whole 16-byte chunks.
#include "launch.h"

namespace jag {

constexpr int kQuantWarps = 8;

__global__ void __launch_bounds__(kQuantWarps * 32)
quantize_kernel(DevIndex ix, int fmt, uint8_t *xq, float *qscale) {
  const int lane = threadIdx.x & 31;
  for (int64_t i = (int64_t)blockIdx.x * kQuantWarps + (threadIdx.x >> 5); i < ix.n;
       i += (int64_t)gridDim.x * kQuantWarps) {
    const float *row = ix.x + i * ix.xs;
    uint8_t *out = xq + i * ix.qbytes;
    if (fmt == JAG_VEC_BF16) {
      for (int j = lane; j < ix.qbytes / 2; j += 32) {
        const uint16_t h = j < ix.d ? __bfloat16_as_ushort(__float2bfloat16_rn(row[j])) : (uint16_t)0;
        reinterpret_cast<uint16_t *>(out)[j] = h;
      }
      if (lane == 0) qscale[i] = 1.f;
    } else {
      float mx = 0.f;
      for (int j = lane; j < ix.d; j += 32) mx = fmaxf(mx, fabsf(row[j]));
#pragma unroll
      for (int o = 16; o >= 1; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, o));
      const float s = mx > 0.f ? __fdiv_rn(mx, 448.f) : 1.f;
      for (int j = lane; j < ix.qbytes; j += 32)
        out[j] = j < ix.d ? (uint8_t)__nv_cvt_float_to_fp8(__fdiv_rn(row[j], s), __NV_SATFINITE, __NV_E4M3) : (uint8_t)0;
      if (lane == 0) qscale[i] = s;
    }
  }
}

cudaError_t quantize_rows(const DevIndex &ix, int fmt, uint8_t *xq, float *qscale, cudaStream_t stream) {
  const int64_t blocks = (ix.n + kQuantWarps - 1) / kQuantWarps;
  quantize_kernel<<<(unsigned)std::min<int64_t>(blocks, 65535), kQuantWarps * 32, 0, stream>>>(ix, fmt, xq, qscale);
  return cudaGetLastError();
}

}  // namespace jag
