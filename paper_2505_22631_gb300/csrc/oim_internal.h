// oim_internal.h -- host-side structures shared by the translation units of liboim.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstdint>
#include <string>
#include <vector>

#include "oim.h"

namespace oim {

// Packed column entry: bit 31 holds the sign of a +-1 weight, the rest the node.
constexpr uint32_t kSignBit = 0x80000000u;

// Per-graph descriptor, readable by kernels.
struct GraphDev {
    int32_t n;          // nodes of this graph
    int32_t node_off;   // first node in the concatenated node arrays
    int32_t edge_off;   // first entry in the concatenated CSR arrays
    int32_t max_deg;    // largest row length
    double  wtot;       // sum_{i<j} w_ij (cut = wtot - agreeing weight)
};

// Schedules and scalars of one launch; K/Ks/Kn point at [graph][steps] arrays.
struct StepParams {
    const float* K;
    const float* Ks;
    const float* Kn;
    int64_t steps;
    float dt;
    float sqrt_dt;
    uint64_t seed;
    const uint64_t* seed_dev;   // when set, kernels read the seed here (CUDA-graph replays
                                // of the per-step forms then serve any seed)
    int32_t q;
    int32_t R;          // replicas
    int32_t R_pad;      // leading dimension of the replica axis
};

// Launch plan of the resident form.
struct ResidentPlan {
    int unit = 4;                  // replicas per thread item: 4 (quad kernel), 2 or 1
    bool csr_smem = false;         // graph structure staged in shared memory
    bool double_buffer = false;    // quad kernel: two (cos, sin) caches, one barrier a step
    int threads = 0;
    size_t smem = 0;
    std::vector<int> k_of_graph;   // replicas per block, per graph
    std::vector<int4> items;       // per block: (graph, first replica, replicas, 0)
};

// Device state of the dense (tensor-core) form of one graph.
struct GemmState {
    int graph = 0;                     // graph of the problem (batch index)
    int n = 0, n_pad = 0, bn = 0, tiles_n = 0;   // n_pad: row length and K extent
    float* theta = nullptr;            // [R_pad][n_pad] phases, replica-major
    void* x[2] = {nullptr, nullptr};   // [2 R_pad][n_pad] bf16 (cos; sin) rows, ping-pong
    void* w = nullptr;                 // [n_pad][n_pad] bf16 coupling matrix
    CUtensorMap map_x[2];
    CUtensorMap map_w;
    // readouts on the tensor cores (q = 2, every weight an integer of magnitude <= 256,
    // exact in BF16): the agreeing weight as (sum_ij w_ij + s^T W s) / 4 for spins s = +-1
    bool score_tc = false;
    CUtensorMap map_w128;              // W in 128-row boxes for the score product
};

struct CSRDev {
    const int32_t* rowp;        // [nodes + 1] global entry offsets
    const uint32_t* col;        // [nnz] global node index, sign bit for +-1 weights
    const float* w;             // [nnz] or nullptr when every |w| == 1
    const int32_t* node_graph;  // [nodes] graph of each node
    const int32_t* split;       // [nodes] first negative-weight entry of each row
    const int32_t* order;       // [nodes] per graph: local node indices by decreasing degree
    const GraphDev* graphs;     // [G]
    int32_t G;
    int32_t nodes;
    // the upper triangle (entries j > i of row i, in row order) for the score passes
    const int32_t* urowp;       // [nodes + 1]
    const uint32_t* ucol;       // packed like col
    const float* uw;            // or nullptr when every |w| == 1
    // [nodes] the stream form's row descriptors {node, row start, first -1 entry, row end},
    // every node of the batch by decreasing row length (stable): the order in which the
    // blocks take their nodes, heaviest rows first
    const int4* srow;
    // [nodes] the first four packed column words of each slot's row, in row order (the
    // slot's own node where the row is shorter: in bounds, never added)
    const uint4* shead;
    // [nodes] row descriptors like srow, graph by graph, heaviest row first within each
    // graph (the adjoint step: a warp's nodes then share a graph for its reductions)
    const int4* arow;
    // [nodes][8] the 16-bit stream form's 32-byte slot descriptors, in srow's order:
    // {node, row start, first -1 entry, row end, graph, local index, first two column
    // indices (the slot's own node where the row is shorter: in bounds, never added)}
    const uint32_t* sdesc;
    // [nnz] column indices without the sign bit (the 16-bit stream form knows a +-1
    // entry's sign from its position against the row's first -1 entry)
    const int32_t* pcol;
    // checked builds (OIM_CHECKS): the word in which the kernels record a column index
    // outside its row's graph (oim_checks.cuh); unused otherwise
    int32_t* check;
};

}  // namespace oim

struct oim_problem_s {
    int32_t q = 2;
    int32_t G = 0;
    int64_t nodes = 0, nnz = 0;
    bool unit_weights = true;      // every |w| == 1: signs packed into col
    bool integer_weights = true;   // every w an integer: exact integer scores
    int device = 0;
    bool uploaded = false;         // device arrays valid
    std::vector<oim::GraphDev> graphs;
    std::vector<int32_t> h_rowp;   // [nodes+1]
    std::vector<uint32_t> h_col;   // [nnz] packed
    std::vector<int32_t> h_col_plain;  // [nnz] global node index
    std::vector<float> h_w;        // [nnz]
    std::vector<int32_t> h_split;  // [nodes] first entry with a negative weight in each row
                                   // (rows hold positive weights first when all |w| == 1)
    std::vector<int32_t> h_order;  // [nodes] local node indices of each graph by decreasing degree
    int32_t* d_rowp = nullptr;
    uint32_t* d_col = nullptr;
    float* d_w = nullptr;
    int32_t* d_node_graph = nullptr;
    int32_t* d_split = nullptr;
    int32_t* d_order = nullptr;
    oim::GraphDev* d_graphs = nullptr;
    int32_t* d_urowp = nullptr;    // upper triangle of the rows (score passes)
    uint32_t* d_ucol = nullptr;
    float* d_uw = nullptr;
    int4* d_srow = nullptr;        // stream-form row descriptors, heaviest rows first
    uint4* d_shead = nullptr;      // and the first four column words of each of those rows
    int4* d_arow = nullptr;        // adjoint row descriptors, graph by graph
    uint32_t* d_sdesc = nullptr;   // 32-byte slot descriptors of the 16-bit stream form
    int32_t* d_pcol = nullptr;     // column indices without sign bits
    int32_t* d_check = nullptr;    // checked builds: index-check word (0: no failure)
    int32_t max_n = 0;             // largest graph
    oim::CSRDev csr() const {
        return oim::CSRDev{d_rowp, d_col, unit_weights ? nullptr : d_w, d_node_graph, d_split,
                           d_order, d_graphs, G, (int32_t)nodes, d_urowp, d_ucol,
                           unit_weights ? nullptr : d_uw, d_srow, d_shead, d_arow, d_sdesc, d_pcol,
                           d_check};
    }
};

struct oim_run_s {
    oim_problem_t p = nullptr;
    int32_t R = 0, R_pad = 0;
    int64_t steps = 0, n_readouts = 0, readout_every = 0;
    uint64_t seed = 0;
    float dt = 0.f;
    oim_run_opts opts{};
    int32_t form = OIM_FORM_STREAM;
    int32_t prec = OIM_PREC_FP32;
    cudaStream_t stream = nullptr;
    int device = 0;
    // device state
    float* d_theta[2] = {nullptr, nullptr};   // [nodes][R_pad]
    void* d_cs[2] = {nullptr, nullptr};       // [nodes][R_pad] (cos, sin) cache
    int final_buf = 0;                        // theta buffer holding the final state
    float* d_sched = nullptr;                 // [3][G][steps_cap]
    int64_t steps_cap = 0;
    int8_t* d_spins = nullptr;                // [nodes][R_pad]
    double* d_trace = nullptr;                // [G][n_readouts_cap][R_pad]
    int64_t readouts_cap = 0;
    double* d_score = nullptr;                // [G][R_pad] scratch for scores
    double* d_energy = nullptr;               // [G][R_pad]
    int32_t* d_err = nullptr;                 // device error word
    uint64_t* d_seed = nullptr;               // the run's seed, read by the per-step forms
    unsigned* d_bar = nullptr;                // persistent form: grid barrier {count, generation}
    // resident-form launch plan
    oim::ResidentPlan plan;
    // dense-form state: the graph of the dense form, or the dense members of a mixed run
    std::vector<oim::GemmState> gemms;
    // mixed runs: the form of each graph, and the stream form's slot descriptors of the
    // CSR members only (sub_slots of them; -1 when the step kernels take every node)
    std::vector<int32_t> graph_forms;
    int4* d_srow_sub = nullptr;
    uint4* d_shead_sub = nullptr;
    uint32_t* d_sdesc_sub = nullptr;
    int32_t sub_slots = -1;
    // with score_split: the node ranges [x, y) whose scores the CSR score pass computes
    // (the graphs not scored on the tensor cores), in node order; otherwise every node
    std::vector<int2> score_ranges;
    bool score_split = false;
    // mixed runs with both parts: the dense members step on a second stream, forked
    // from the run's stream after each readout and joined before the next one
    cudaStream_t aux = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // stream form: the scoring half of each readout runs on a second stream beside the
    // next steps (it reads only the spins, which the steps do not touch)
    cudaStream_t aux_score = nullptr;
    cudaEvent_t ev_spins = nullptr, ev_scored = nullptr;
    int4* d_items = nullptr;                  // plan.items on the device
    // stream-form CUDA graph of a whole run, reused while its shape is unchanged
    cudaGraphExec_t chunk_exec = nullptr;
    int64_t graph_steps = -1;
    float graph_dt = 0.f;
    int64_t seen_steps = -1;                  // shape of the last direct execution
    float seen_dt = 0.f;
    // a replayable chunk of steps (step base in d_t0) for first executions
    cudaGraphExec_t step_chunk_exec = nullptr;
    int64_t step_chunk_len = 0;
    float step_chunk_dt = 0.f;
    int64_t step_chunk_every = -1;
    int32_t* d_t0 = nullptr;                  // device step counter (graph replays)
    // adjoint support: phases every ckpt_every steps ([n_ckpt][nodes][R_pad])
    int32_t ckpt_every = 0;
    int64_t ckpt_cap = 0;
    float* d_ckpt = nullptr;
    // ckpt_every 1, when it fits in device memory: the coupling sums (A, B) of every
    // step as well ([steps][nodes][R_pad]), so the backward pass recomputes nothing
    float2* d_ab = nullptr;
    int64_t ab_cap = 0;                       // steps the buffer was sized (or tried) for
    bool ran = false;
};

namespace oim {

// Makes a device current for the lifetime of the object and gives the calling thread
// its previous current device back when the object goes out of scope, so that no entry
// point leaves a multi-device caller switched to another GPU.
class DeviceScope {
public:
    DeviceScope() = default;
    DeviceScope(const DeviceScope&) = delete;
    DeviceScope& operator=(const DeviceScope&) = delete;
    cudaError_t enter(int device) {
        int cur = -1;
        cudaError_t e = cudaGetDevice(&cur);
        if (e != cudaSuccess) return e;
        if (cur == device) return cudaSuccess;
        e = cudaSetDevice(device);
        if (e == cudaSuccess) {
            prev_ = cur;
            switched_ = true;
        }
        return e;
    }
    ~DeviceScope() {
        if (switched_) cudaSetDevice(prev_);
    }

private:
    int prev_ = -1;
    bool switched_ = false;
};

// A named range on the profiler's timeline for the lifetime of the object (NVTX; a no-op
// unless a tool is attached).
class NvtxRange {
public:
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// the autotuner's cached choice for a problem shape and replica count (false if none)
bool cached_choice(const oim_problem_s* p, int32_t replicas, oim_run_opts* out);

// error reporting (thread-local message)
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);

// The graph structure as the step kernels of run r see it: every node of the problem,
// or in a mixed run only the slots of its CSR members.
inline CSRDev step_csr(const oim_run_s& r) {
    CSRDev c = r.p->csr();
    if (r.sub_slots >= 0) {
        c.srow = r.d_srow_sub;
        c.shead = r.d_shead_sub;
        c.sdesc = r.d_sdesc_sub;
        c.nodes = r.sub_slots;
    }
    return c;
}

// launchers (return cudaError_t of the launch)
cudaError_t launch_init_stream(const oim_run_s& r, cudaStream_t s);
cudaError_t launch_step_stream(const oim_run_s& r, int64_t t, const int32_t* d_t0, cudaStream_t s);
cudaError_t launch_persistent_steps(const oim_run_s& r, int64_t t0, int64_t t1, cudaStream_t s);
cudaError_t plan_resident(const oim_problem_s& p, int32_t R_pad, int32_t prec, int32_t want_k,
                          int32_t want_threads, ResidentPlan* plan);

}  // namespace oim
