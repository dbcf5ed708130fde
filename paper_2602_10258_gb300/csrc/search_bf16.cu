// Graph-search kernels for rows stored as bf16.
#include "query_graph.cuh"

namespace jag {
template cudaError_t launch_graph_fmt<JAG_VEC_BF16>(const SearchLaunch &L);
}  // namespace jag
