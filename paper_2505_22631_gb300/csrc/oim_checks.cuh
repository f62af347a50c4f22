// oim_checks.cuh -- index checks of the checked build.
//
// Built with -DOIM_CHECKS (build(checks=True), liboim_checks.so), every kernel that
// gathers by column index tests the index against the node range of the row's graph
// before it uses it; an index outside that range is recorded in the problem's check
// word (CSRDev::check, read back by oim_run_sync as OIM_EINDEX) and replaced by a node
// of the row's own graph, so the kernel never reads outside its buffers.  The other
// builds compile the checks away.
#pragma once

#include "oim_internal.h"

namespace oim {

#ifdef OIM_CHECKS
constexpr bool kChecks = true;
#else
constexpr bool kChecks = false;
#endif

constexpr int32_t kCheckIndex = 1;

__device__ __forceinline__ void record_check(const CSRDev& csr) {
    if (csr.check) atomicOr(csr.check, kCheckIndex);
}

// Global node index j of an entry of a row of graph g: j itself when it is a node of g,
// else `fallback` (a node of g, e.g. the row's own) with the failure recorded.
__device__ __forceinline__ uint32_t checked_node(const CSRDev& csr, int g, uint32_t j, uint32_t fallback) {
    if constexpr (kChecks) {
        const GraphDev gd = csr.graphs[g];
        if (j - (uint32_t)gd.node_off >= (uint32_t)gd.n) {
            record_check(csr);
            return fallback;
        }
    }
    return j;
}

// The same for a row whose graph is not at hand: the row's node names it.
__device__ __forceinline__ uint32_t checked_node_of_row(const CSRDev& csr, int row_node, uint32_t j) {
    if constexpr (kChecks) return checked_node(csr, csr.node_graph[row_node], j, (uint32_t)row_node);
    return j;
}

// Local node index jl (0 <= jl < n) of an entry of a graph of n nodes.
__device__ __forceinline__ int checked_local(const CSRDev& csr, int n, int jl, int fallback) {
    if constexpr (kChecks) {
        if ((unsigned)jl >= (unsigned)n) {
            record_check(csr);
            return fallback;
        }
    }
    return jl;
}

}  // namespace oim
