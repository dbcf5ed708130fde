// Launch of the serve loop for one row format: picks the lane mapping of the
// stored rows and of the fp32 rows, sizes the persistent grid to what is
// resident at once (every CTA must run concurrently: the loop's CTAs only
// leave through their own bounded waits).
#pragma once

#include "launch.h"
#include "launch_util.cuh"
#include "serve_core.cuh"

namespace jag {

template <int P, int CPL, int FMT, bool POL, int CPLF>
static cudaError_t launch_serve_one(const ServeArgs &a, int ctas, cudaStream_t stream, int *grid_out) {
  const size_t smem = (size_t)kSearchWarps * warp_smem_bytes(list_slots(a.ls), a.hbits);
  auto kern = serve_kernel<256, P, CPL, FMT, POL, CPLF>;
  const int bps = blocks_per_sm(kern, smem);
  if (bps == 0) return cudaErrorInvalidConfiguration;
  const int resident = bps * num_sms();
  const int grid = ctas > 0 && ctas < resident ? ctas : resident;
  kern<<<grid, kSearchWarps * 32, smem, stream>>>(a);
  *grid_out = grid;
  return cudaGetLastError();
}

template <int P, int CPL, int FMT, int CPLF>
static cudaError_t launch_serve_pol(const ServeArgs &a, int ctas, cudaStream_t stream, int *grid_out) {
  if (a.has_policy) return launch_serve_one<P, CPL, FMT, true, CPLF>(a, ctas, stream, grid_out);
  return launch_serve_one<P, CPL, FMT, false, CPLF>(a, ctas, stream, grid_out);
}

template <int FMT>
cudaError_t launch_serve_fmt(const ServeArgs &a, int ctas, cudaStream_t stream, int *grid_out) {
  int P, CPL, PF, CPLF;
  const int nch = FMT == JAG_VEC_F32 ? a.ix.nchunks : a.ix.qchunks;
  if (!row_mapping(nch, &P, &CPL) || !row_mapping(a.ix.nchunks, &PF, &CPLF)) return cudaErrorInvalidValue;
  // the exact scan and the re-rank use all 32 lanes per fp32 row
  if (a.ix.nchunks > 64) return cudaErrorInvalidValue;
  CPLF = a.ix.nchunks <= 32 ? 1 : 2;
  if constexpr (FMT == JAG_VEC_F32) {
    if (P == 8) return launch_serve_pol<8, 1, FMT, 1>(a, ctas, stream, grid_out);
    if (P == 16) return launch_serve_pol<16, 1, FMT, 1>(a, ctas, stream, grid_out);
    if (CPL == 1) return launch_serve_pol<32, 1, FMT, 1>(a, ctas, stream, grid_out);
    if (CPL == 2) return launch_serve_pol<32, 2, FMT, 2>(a, ctas, stream, grid_out);
  } else {
    if (CPL != 1) return cudaErrorInvalidValue;
#define JAG_SCASE(PP)                                                                \
  if (P == PP) {                                                                     \
    if (CPLF == 1) return launch_serve_pol<PP, 1, FMT, 1>(a, ctas, stream, grid_out); \
    return launch_serve_pol<PP, 1, FMT, 2>(a, ctas, stream, grid_out);               \
  }
    JAG_SCASE(8)
    JAG_SCASE(16)
    JAG_SCASE(32)
#undef JAG_SCASE
  }
  return cudaErrorInvalidValue;
}

}  // namespace jag
