// Graph-search kernels for rows stored as f32.
#include "query_graph.cuh"

namespace jag {
template cudaError_t launch_graph_fmt<JAG_VEC_F32>(const SearchLaunch &L);
}  // namespace jag
