// Graph-search kernels for rows stored as fp8.
#include "query_graph.cuh"

namespace jag {
template cudaError_t launch_graph_fmt<JAG_VEC_FP8>(const SearchLaunch &L);
}  // namespace jag
