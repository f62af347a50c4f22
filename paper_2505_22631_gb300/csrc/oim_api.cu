// oim_api.cu -- the C ABI of liboim (declared in include/oim.h): argument
// validation, device allocation, choice of the integration form and the launch
// sequence of a run.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "oim_internal.h"

namespace oim {

static thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
    g_last_error = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? OIM_ENOMEM : OIM_ECUDA;
}

// implemented in the kernel translation units
cudaError_t launch_score(const oim_run_s& r, const float* theta, int64_t k, cudaStream_t s);
cudaError_t launch_spins(const oim_run_s& r, const float* theta, cudaStream_t s);
cudaError_t launch_score_pass(const oim_run_s& r, int64_t k, const int32_t* d_t0, int32_t t_add, cudaStream_t s);
cudaError_t launch_score_at(const oim_run_s& r, const float* theta, int64_t k, const int32_t* d_t0,
                            int32_t t_add, cudaStream_t s);
cudaError_t launch_finalize(const oim_run_s& r, int64_t k, double* score, cudaStream_t s);
cudaError_t launch_energy_of(const oim_run_s& r, const float* theta, double* energy, cudaStream_t s);
cudaError_t launch_gather(const oim_run_s& r, const float* theta, int8_t* spins, float* th_out,
                          cudaStream_t s);
cudaError_t launch_resident_impl(const oim_run_s& r, const int4* d_items, cudaStream_t s);
cudaError_t launch_derivative(const oim_problem_s& p, const float* theta, int32_t R, float K,
                              float Ks, float* f, cudaStream_t s);
size_t resident_cache_bytes(int32_t prec);
cudaError_t launch_cs_from_theta(const oim_run_s& r, const float* theta, float2* cs, cudaStream_t s);
cudaError_t launch_step_stream_buffers(const oim_run_s& r, int64_t t, const float* th_in,
                                       const float2* cs_in, float* th_out, float2* cs_out, float2* ab,
                                       cudaStream_t s);
int gemm_setup(oim_run_s& r, int graph);
void gemm_free(oim_run_s& r);
cudaError_t launch_gemm_init(const oim_run_s& r, int k, cudaStream_t s);
cudaError_t launch_set_seed(uint64_t* d_seed, uint64_t seed, cudaStream_t s);
cudaError_t launch_gemm_step_at(const oim_run_s& r, int k, int64_t t, const int32_t* d_t0, cudaStream_t s);
cudaError_t launch_gemm_to_common(const oim_run_s& r, int k, float* out, cudaStream_t s);
cudaError_t launch_gemm_score(const oim_run_s& r, int k, int64_t k_slot, const int32_t* d_t0, int32_t t_add,
                              int xbuf, cudaStream_t s);

// dense state k is scored on the tensor cores at readouts
inline bool tc_scored(const oim_run_s& r, int k) { return r.score_split && r.gemms[(size_t)k].score_tc; }
cudaError_t launch_adj_planes(const oim_run_s& r, const float* theta, const float* lam, float* Y,
                              cudaStream_t s);
cudaError_t launch_adj_terminal(const oim_run_s& r, const float* Y, float* lam, double* loss, cudaStream_t s);
cudaError_t launch_adj_step(const oim_run_s& r, int64_t t, const float* theta, const float* theta_prev,
                            const float2* AB, const float* Ylam, float* Ylam_out, const float* lam_in,
                            float* lam_out, double* dK, double* dKs, double* dKn, cudaStream_t s);

}  // namespace oim

using namespace oim;

#define OIM_CUDA(call, what)                          \
    do {                                              \
        cudaError_t e__ = (call);                     \
        if (e__ != cudaSuccess) return cuda_fail(e__, what); \
    } while (0)

namespace {

template <typename T>
cudaError_t dev_alloc(T** p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    return cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T));
}

template <typename T>
void dev_free(T*& p) {
    if (p) cudaFree(p);
    p = nullptr;
}

// True when p is device (or managed) memory.  Without a usable driver every
// pointer is taken as host memory, so argument validation runs anywhere.
bool is_device_ptr(const void* p) {
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

// copy count elements from host or device memory into a host vector
template <typename T>
cudaError_t fetch(std::vector<T>& out, const T* src, size_t count) {
    out.resize(count);
    if (count == 0) return cudaSuccess;
    if (!is_device_ptr(src)) {
        std::memcpy(out.data(), src, count * sizeof(T));
        return cudaSuccess;
    }
    return cudaMemcpy(out.data(), src, count * sizeof(T), cudaMemcpyDeviceToHost);
}

// A read-only view of a caller's array: the array itself when it is host memory, else
// a host copy of it in `store`.
template <typename T>
cudaError_t view(const T*& out, std::vector<T>& store, const T* src, size_t count) {
    out = src;
    if (count == 0 || !is_device_ptr(src)) return cudaSuccess;
    const cudaError_t e = fetch(store, src, count);
    out = store.data();
    return e;
}

// fn(k) for every k in [0, count), on up to kHostThreads host threads (the calling
// thread among them) taking items in order from a shared counter; on the calling thread
// alone when the work (entries to touch) is small or no thread can be started.  fn must
// not throw.
constexpr int kHostThreads = 16;
constexpr int64_t kParallelWork = 1 << 20;

template <typename F>
void parallel_for(int64_t count, int64_t work, F&& fn) {
    const unsigned hw = std::thread::hardware_concurrency();
    int64_t threads = std::min<int64_t>(count, std::min<int64_t>(kHostThreads, hw ? (int64_t)hw : 1));
    if (work < kParallelWork) threads = 1;
    std::atomic<int64_t> next{0};
    auto worker = [&]() {
        for (int64_t k = next.fetch_add(1); k < count; k = next.fetch_add(1)) fn(k);
    };
    std::vector<std::thread> pool;
    try {
        for (int64_t t = 1; t < threads; ++t) pool.emplace_back(worker);
    } catch (...) {
        // fewer threads than asked (the items are shared out all the same)
    }
    worker();
    for (auto& th : pool) th.join();
}

void free_problem(oim_problem_s* p);

// The stream form's slot descriptors for the nodes of the graphs with take[g] set,
// heaviest row first (a stable sort by row length, so a subset keeps the order it has
// among all nodes): srow {node, row start, first -1 entry, row end}; shead, the first
// four packed column words; sdesc (32 bytes) {node, row start, first -1 entry, row end,
// graph, local index, first two column indices}.  Rows shorter than the heads are
// padded with the slot's own node (in bounds, never added).
struct StreamSlots {
    std::vector<int4> srow;
    std::vector<uint4> shead;
    std::vector<uint32_t> sdesc;
};

StreamSlots build_stream_slots(const oim_problem_s* p, const std::vector<char>& take) {
    std::vector<int32_t> node_g((size_t)p->nodes);
    std::vector<int32_t> order;
    for (int g = 0; g < p->G; ++g)
        for (int32_t k = 0; k < p->graphs[g].n; ++k) {
            const int32_t v = p->graphs[g].node_off + k;
            node_g[(size_t)v] = g;
            if (take[(size_t)g]) order.push_back(v);
        }
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
        return p->h_rowp[a + 1] - p->h_rowp[a] > p->h_rowp[b + 1] - p->h_rowp[b];
    });
    StreamSlots sl;
    sl.srow.resize(order.size());
    sl.shead.resize(order.size());
    sl.sdesc.resize(order.size() * 8);
    for (size_t k = 0; k < order.size(); ++k) {
        const int32_t v = order[k];
        const int g = node_g[(size_t)v];
        sl.srow[k] = make_int4(v, p->h_rowp[v], p->h_split[v], p->h_rowp[v + 1]);
        uint32_t h[4];
        for (int u = 0; u < 4; ++u) {
            const int64_t e = (int64_t)p->h_rowp[v] + u;
            h[u] = e < p->h_rowp[v + 1] ? p->h_col[(size_t)e] : (uint32_t)v;
        }
        sl.shead[k] = make_uint4(h[0], h[1], h[2], h[3]);
        uint32_t* d = sl.sdesc.data() + 8 * k;
        d[0] = (uint32_t)v;
        d[1] = (uint32_t)p->h_rowp[v];
        d[2] = (uint32_t)p->h_split[v];
        d[3] = (uint32_t)p->h_rowp[v + 1];
        d[4] = (uint32_t)g;
        d[5] = (uint32_t)(v - p->graphs[g].node_off);
        for (int u = 0; u < 2; ++u) {
            const int64_t e = (int64_t)p->h_rowp[v] + u;
            d[6 + u] = e < p->h_rowp[v + 1] ? (uint32_t)p->h_col_plain[(size_t)e] : (uint32_t)v;
        }
    }
    return sl;
}

cudaError_t upload_stream_slots(const StreamSlots& sl, int4* srow, uint4* shead, uint32_t* sdesc) {
    if (sl.srow.empty()) return cudaSuccess;
    cudaError_t e = cudaMemcpy(srow, sl.srow.data(), sl.srow.size() * sizeof(int4), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(shead, sl.shead.data(), sl.shead.size() * sizeof(uint4), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(sdesc, sl.sdesc.data(), sl.sdesc.size() * sizeof(uint32_t), cudaMemcpyHostToDevice);
    return e;
}

int upload_problem(oim_problem_s* p) {
    OIM_CUDA(dev_alloc(&p->d_rowp, p->h_rowp.size()), "cudaMalloc(row_ptr)");
    OIM_CUDA(dev_alloc(&p->d_col, p->h_col.size()), "cudaMalloc(col)");
    // (+-1 weights: the kernels take the sign from the packed columns and never read w)
    OIM_CUDA(dev_alloc(&p->d_w, p->unit_weights ? 1 : p->h_w.size()), "cudaMalloc(w)");
    OIM_CUDA(dev_alloc(&p->d_node_graph, (size_t)p->nodes), "cudaMalloc(node_graph)");
    OIM_CUDA(dev_alloc(&p->d_split, (size_t)p->nodes), "cudaMalloc(split)");
    OIM_CUDA(dev_alloc(&p->d_order, (size_t)p->nodes), "cudaMalloc(order)");
    OIM_CUDA(dev_alloc(&p->d_graphs, p->graphs.size()), "cudaMalloc(graphs)");
    // the stream form's blocks take nodes heaviest rows first across the whole batch, so
    // the blocks that run last are the short ones (longest-processing-time-first order);
    // each slot's row bounds travel with the node in its descriptors
    {
        StreamSlots sl = build_stream_slots(p, std::vector<char>((size_t)p->G, 1));
        OIM_CUDA(dev_alloc(&p->d_srow, sl.srow.size()), "cudaMalloc(stream rows)");
        OIM_CUDA(dev_alloc(&p->d_shead, sl.shead.size()), "cudaMalloc(stream row heads)");
        OIM_CUDA(dev_alloc(&p->d_sdesc, sl.sdesc.size()), "cudaMalloc(stream slot descriptors)");
        OIM_CUDA(upload_stream_slots(sl, p->d_srow, p->d_shead, p->d_sdesc), "upload stream slots");
        OIM_CUDA(dev_alloc(&p->d_pcol, p->h_col_plain.size()), "cudaMalloc(plain columns)");
        if (!p->h_col_plain.empty())
            OIM_CUDA(cudaMemcpy(p->d_pcol, p->h_col_plain.data(), p->h_col_plain.size() * 4,
                                cudaMemcpyHostToDevice),
                     "upload plain columns");
    }
    // the adjoint's descriptors: graph by graph, each graph's rows by decreasing length
    OIM_CUDA(dev_alloc(&p->d_arow, (size_t)p->nodes), "cudaMalloc(adjoint rows)");
    std::vector<int4> arow((size_t)p->nodes);
    for (int g = 0; g < p->G; ++g) {
        const int32_t off = p->graphs[g].node_off;
        for (int32_t k = 0; k < p->graphs[g].n; ++k) {
            const int32_t v = off + p->h_order[(size_t)off + k];
            arow[(size_t)off + k] = make_int4(v, p->h_rowp[v], p->h_split[v], p->h_rowp[v + 1]);
        }
    }
    OIM_CUDA(cudaMemcpy(p->d_arow, arow.data(), arow.size() * sizeof(int4), cudaMemcpyHostToDevice),
             "upload adjoint rows");
    std::vector<int32_t> ng((size_t)p->nodes);
    for (int g = 0; g < p->G; ++g)
        std::fill(ng.begin() + p->graphs[g].node_off,
                  ng.begin() + p->graphs[g].node_off + p->graphs[g].n, g);
    OIM_CUDA(cudaMemcpy(p->d_rowp, p->h_rowp.data(), p->h_rowp.size() * 4, cudaMemcpyHostToDevice),
             "upload row_ptr");
    if (!p->h_col.empty())
        OIM_CUDA(cudaMemcpy(p->d_col, p->h_col.data(), p->h_col.size() * 4, cudaMemcpyHostToDevice),
                 "upload col");
    if (!p->h_w.empty() && !p->unit_weights)
        OIM_CUDA(cudaMemcpy(p->d_w, p->h_w.data(), p->h_w.size() * 4, cudaMemcpyHostToDevice),
                 "upload w");
    OIM_CUDA(cudaMemcpy(p->d_node_graph, ng.data(), ng.size() * 4, cudaMemcpyHostToDevice),
             "upload node_graph");
    OIM_CUDA(cudaMemcpy(p->d_split, p->h_split.data(), p->h_split.size() * 4, cudaMemcpyHostToDevice),
             "upload split");
    OIM_CUDA(cudaMemcpy(p->d_order, p->h_order.data(), p->h_order.size() * 4, cudaMemcpyHostToDevice),
             "upload order");
    OIM_CUDA(cudaMemcpy(p->d_graphs, p->graphs.data(), p->graphs.size() * sizeof(GraphDev),
                        cudaMemcpyHostToDevice),
             "upload graphs");
    // the upper triangle of every row, in row order, for the score passes (counted, then
    // filled, graph by graph on host threads)
    std::vector<int32_t> urowp((size_t)p->nodes + 1, 0);
    parallel_for(p->G, p->nnz, [&](int64_t g) {
        const int64_t i0 = p->graphs[(size_t)g].node_off, i1 = i0 + p->graphs[(size_t)g].n;
        for (int64_t i = i0; i < i1; ++i) {
            int32_t c = 0;
            for (int32_t e = p->h_rowp[i]; e < p->h_rowp[i + 1]; ++e) c += p->h_col_plain[e] > i;
            urowp[(size_t)i + 1] = c;
        }
    });
    for (int64_t i = 0; i < p->nodes; ++i) urowp[(size_t)i + 1] += urowp[(size_t)i];
    std::vector<uint32_t> ucol((size_t)urowp[(size_t)p->nodes]);
    std::vector<float> uw(p->unit_weights ? 0 : ucol.size());
    parallel_for(p->G, p->nnz, [&](int64_t g) {
        const int64_t i0 = p->graphs[(size_t)g].node_off, i1 = i0 + p->graphs[(size_t)g].n;
        for (int64_t i = i0; i < i1; ++i) {
            int32_t at = urowp[(size_t)i];
            for (int32_t e = p->h_rowp[i]; e < p->h_rowp[i + 1]; ++e) {
                if (p->h_col_plain[e] <= i) continue;
                ucol[(size_t)at] = p->h_col[e];
                if (!p->unit_weights) uw[(size_t)at] = p->h_w[e];
                ++at;
            }
        }
    });
    OIM_CUDA(dev_alloc(&p->d_urowp, urowp.size()), "cudaMalloc(upper row_ptr)");
    OIM_CUDA(dev_alloc(&p->d_ucol, std::max<size_t>(ucol.size(), 1)), "cudaMalloc(upper col)");
    OIM_CUDA(dev_alloc(&p->d_uw, std::max<size_t>(uw.size(), 1)), "cudaMalloc(upper w)");
    OIM_CUDA(cudaMemcpy(p->d_urowp, urowp.data(), urowp.size() * 4, cudaMemcpyHostToDevice),
             "upload upper row_ptr");
    if (!ucol.empty())
        OIM_CUDA(cudaMemcpy(p->d_ucol, ucol.data(), ucol.size() * 4, cudaMemcpyHostToDevice),
                 "upload upper col");
    if (!uw.empty())
        OIM_CUDA(cudaMemcpy(p->d_uw, uw.data(), uw.size() * 4, cudaMemcpyHostToDevice), "upload upper w");
    OIM_CUDA(dev_alloc(&p->d_check, 1), "cudaMalloc(check word)");
    OIM_CUDA(cudaMemset(p->d_check, 0, sizeof(int32_t)), "clear check word");
    p->uploaded = true;
    return OIM_OK;
}

int ensure_uploaded(oim_problem_s* p) {
    if (p->uploaded) return OIM_OK;
    int rc = upload_problem(p);
    if (rc != OIM_OK) free_problem(p);
    return rc;
}

void free_problem(oim_problem_s* p) {
    p->uploaded = false;
    dev_free(p->d_rowp);
    dev_free(p->d_col);
    dev_free(p->d_w);
    dev_free(p->d_node_graph);
    dev_free(p->d_split);
    dev_free(p->d_order);
    dev_free(p->d_srow);
    dev_free(p->d_shead);
    dev_free(p->d_arow);
    dev_free(p->d_sdesc);
    dev_free(p->d_pcol);
    dev_free(p->d_graphs);
    dev_free(p->d_urowp);
    dev_free(p->d_ucol);
    dev_free(p->d_uw);
    dev_free(p->d_check);
}

void free_run_buffers(oim_run_s* r) {
    if (r->d_theta[1] == r->d_theta[0]) r->d_theta[1] = nullptr;   // the stream form's alias
    dev_free(r->d_theta[0]);
    dev_free(r->d_theta[1]);
    if (r->d_cs[0]) cudaFree(r->d_cs[0]);
    if (r->d_cs[1]) cudaFree(r->d_cs[1]);
    r->d_cs[0] = r->d_cs[1] = nullptr;
    dev_free(r->d_sched);
    dev_free(r->d_spins);
    dev_free(r->d_trace);
    dev_free(r->d_score);
    dev_free(r->d_energy);
    dev_free(r->d_err);
    dev_free(r->d_seed);
    dev_free(r->d_t0);
    dev_free(r->d_bar);
    dev_free(r->d_items);
    dev_free(r->d_ckpt);
    dev_free(r->d_ab);
    r->ab_cap = 0;
    dev_free(r->d_srow_sub);
    dev_free(r->d_shead_sub);
    dev_free(r->d_sdesc_sub);
    r->sub_slots = -1;
    r->score_ranges.clear();
    r->score_split = false;
    if (r->aux) cudaStreamDestroy(r->aux);
    if (r->ev_fork) cudaEventDestroy(r->ev_fork);
    if (r->ev_join) cudaEventDestroy(r->ev_join);
    r->aux = nullptr;
    r->ev_fork = r->ev_join = nullptr;
    if (r->aux_score) cudaStreamDestroy(r->aux_score);
    if (r->ev_spins) cudaEventDestroy(r->ev_spins);
    if (r->ev_scored) cudaEventDestroy(r->ev_scored);
    r->aux_score = nullptr;
    r->ev_spins = r->ev_scored = nullptr;
    gemm_free(*r);
    if (r->chunk_exec) cudaGraphExecDestroy(r->chunk_exec);
    r->chunk_exec = nullptr;
    if (r->step_chunk_exec) cudaGraphExecDestroy(r->step_chunk_exec);
    r->step_chunk_exec = nullptr;
}

int validate_schedule_args(float dt, int64_t steps) {
    if (!(dt > 0.f) || !std::isfinite(dt)) return fail(OIM_EINVAL, "dt must be finite and > 0");
    if (steps < 0 || steps >= ((int64_t)1 << 32)) return fail(OIM_EINVAL, "steps out of range");
    return OIM_OK;
}

// Captured graphs hold the buffer pointers and strides of the run: any reallocation
// below drops them (they are captured again when needed).
static void drop_graphs(oim_run_s* r) {
    if (r->chunk_exec) cudaGraphExecDestroy(r->chunk_exec);
    r->chunk_exec = nullptr;
    r->graph_steps = -1;
    if (r->step_chunk_exec) cudaGraphExecDestroy(r->step_chunk_exec);
    r->step_chunk_exec = nullptr;
    r->step_chunk_len = 0;
}

// (Re)allocate the buffers whose size depends on steps / readouts.
int ensure_step_buffers(oim_run_s* r, int64_t steps) {
    const int G = r->p->G;
    const int64_t n_ro = r->readout_every > 0 ? steps / r->readout_every : 0;
    if (steps > r->steps_cap || !r->d_sched) {
        drop_graphs(r);
        dev_free(r->d_sched);
        r->steps_cap = std::max<int64_t>(steps, 1);
        OIM_CUDA(dev_alloc(&r->d_sched, (size_t)3 * G * r->steps_cap), "cudaMalloc(schedules)");
    }
    if (r->ckpt_every > 0) {
        const int64_t need = steps / r->ckpt_every + 1;
        if (need > r->ckpt_cap || !r->d_ckpt) {
            drop_graphs(r);
            dev_free(r->d_ckpt);
            r->ckpt_cap = need;
            OIM_CUDA(dev_alloc(&r->d_ckpt, (size_t)need * r->p->nodes * r->R_pad), "cudaMalloc(checkpoints)");
        }
    }
    if (r->ckpt_every == 1 && steps > r->ab_cap) {
        // the whole trajectory's coupling sums, 8 B per node-replica-step, when they fit
        // with a tenth of the device (at least 2 GiB) left over; otherwise the backward
        // pass recomputes them step by step
        drop_graphs(r);
        dev_free(r->d_ab);
        r->ab_cap = steps;
        const size_t bytes = (size_t)steps * r->p->nodes * r->R_pad * sizeof(float2);
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess &&
            bytes + std::max<size_t>(total_b / 10, (size_t)2 << 30) <= free_b) {
            if (cudaMalloc(&r->d_ab, bytes) != cudaSuccess) r->d_ab = nullptr;
        }
        cudaGetLastError();
    }
    const int64_t ro_need = n_ro + 1;   // one extra row for the final scores
    if (ro_need > r->readouts_cap || !r->d_trace) {
        drop_graphs(r);
        dev_free(r->d_trace);
        r->readouts_cap = ro_need;
        OIM_CUDA(dev_alloc(&r->d_trace, (size_t)G * r->readouts_cap * r->R_pad), "cudaMalloc(trace)");
    }
    return OIM_OK;
}

int choose_form(oim_run_s* r) {
    int form = r->opts.form;
    int prec = r->opts.precision;
    if (form < OIM_FORM_AUTO || form > OIM_FORM_PERSISTENT) return fail(OIM_EINVAL, "unknown form");
    if (form == OIM_FORM_PERSISTENT) {
        if (r->opts.checkpoint_every > 0)
            return fail(OIM_EUNSUPPORTED, "checkpoints (for oim_backward) need the FP32 stream form");
        if (prec == OIM_PREC_FP32)
            return fail(OIM_EUNSUPPORTED, "the persistent form keeps a 16-bit (cos, sin) cache");
        int dev = 0, coop = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) {
            cudaGetLastError();
            return fail(OIM_EUNSUPPORTED, "the device does not support cooperative launches");
        }
        r->form = OIM_FORM_PERSISTENT;
        r->prec = prec == OIM_PREC_AUTO ? OIM_PREC_FP16 : prec;
        r->R_pad = (r->R + 7) & ~7;   // octets of replicas
        return OIM_OK;
    }
    if (prec < OIM_PREC_AUTO || prec > OIM_PREC_FP16) return fail(OIM_EINVAL, "unknown precision");
    if (form == OIM_FORM_MIXED) {
        // graph_forms names each graph's form: the CSR members step together in the
        // stream form with the cache precision asked for (FP16 by default), each dense
        // member on the tensor cores (BF16 operands)
        if (!r->opts.graph_forms) return fail(OIM_EINVAL, "OIM_FORM_MIXED needs graph_forms");
        if (r->opts.checkpoint_every > 0)
            return fail(OIM_EUNSUPPORTED, "checkpoints (for oim_backward) need the FP32 stream form");
        if (r->opts.threads_per_block != 0 && r->opts.threads_per_block != 320 &&
            r->opts.threads_per_block != 576)
            return fail(OIM_EINVAL, "mixed form: threads_per_block is 0, 320 or 576 (the dense members' tiles)");
        r->graph_forms.assign(r->opts.graph_forms, r->opts.graph_forms + r->p->G);
        bool dense = false;
        for (int32_t f : r->graph_forms) {
            if (f != OIM_FORM_STREAM && f != OIM_FORM_GEMM)
                return fail(OIM_EINVAL, "graph_forms entries are OIM_FORM_STREAM or OIM_FORM_GEMM");
            dense |= f == OIM_FORM_GEMM;
        }
        r->form = OIM_FORM_MIXED;
        r->prec = prec == OIM_PREC_AUTO ? OIM_PREC_FP16 : prec;
        // X^T tiles hold 64 replicas; the 16-bit stream form moves octets
        r->R_pad = dense ? (r->R + 63) & ~63 : (r->prec == OIM_PREC_FP32 ? (r->R + 3) & ~3 : (r->R + 7) & ~7);
        return OIM_OK;
    }
    if (form == OIM_FORM_GEMM) {
        if (r->p->G != 1) return fail(OIM_EUNSUPPORTED, "the dense form takes one graph per run");
        if (prec != OIM_PREC_AUTO && prec != OIM_PREC_BF16)
            return fail(OIM_EUNSUPPORTED, "the dense form multiplies BF16 operands");
        if (r->opts.checkpoint_every > 0)
            return fail(OIM_EUNSUPPORTED, "checkpoints (for oim_backward) need the FP32 stream form");
        if (r->opts.threads_per_block != 0 && r->opts.threads_per_block != 320 &&
            r->opts.threads_per_block != 576)
            return fail(OIM_EINVAL, "dense form: threads_per_block is 0, 320 (128-wide tiles) or 576 "
                                    "(256-wide tiles)");
        r->form = OIM_FORM_GEMM;
        r->prec = OIM_PREC_BF16;
        r->R_pad = (r->R + 63) & ~63;    // X^T tiles hold 64 replicas (128 rows)
        return OIM_OK;
    }
    if (r->opts.checkpoint_every < 0) return fail(OIM_EINVAL, "checkpoint_every must be >= 0");
    if (r->opts.checkpoint_every > 0) {
        // the adjoint recomputes segments with the stream kernels: the forward uses them too
        if (form == OIM_FORM_RESIDENT || (prec != OIM_PREC_AUTO && prec != OIM_PREC_FP32))
            return fail(OIM_EUNSUPPORTED, "checkpoints (for oim_backward) need the FP32 stream form");
        form = OIM_FORM_STREAM;
        prec = OIM_PREC_FP32;
    }
    // AUTO precision: the resident form keeps its (cos, sin) cache in FP16 (twice
    // the replicas per block of FP32, coupling error ~1e-4 relative); the stream
    // form defaults to FP32 (the plain form) and takes FP16 / BF16 when asked.
    if (prec == OIM_PREC_AUTO) prec = (form == OIM_FORM_STREAM) ? OIM_PREC_FP32 : OIM_PREC_FP16;
    if (form == OIM_FORM_AUTO && r->opts.precision == OIM_PREC_AUTO && r->opts.checkpoint_every == 0 &&
        r->opts.replicas_per_block == 0 && r->opts.threads_per_block == 0) {
        // a shape the autotuner has timed in this process takes its choice
        oim_run_opts tuned;
        if (cached_choice(r->p, r->R, &tuned)) {
            r->opts.form = tuned.form;
            r->opts.precision = tuned.precision;
            r->opts.replicas_per_block = tuned.replicas_per_block;
            r->opts.threads_per_block = tuned.threads_per_block;
            r->opts.graph_forms = tuned.graph_forms;
            return choose_form(r);
        }
    }
    if (form == OIM_FORM_AUTO) {
        ResidentPlan tmp;
        form = plan_resident(*r->p, r->R_pad, prec, r->opts.replicas_per_block,
                             r->opts.threads_per_block, &tmp) == cudaSuccess
                   ? OIM_FORM_RESIDENT
                   : OIM_FORM_STREAM;
        if (form == OIM_FORM_STREAM && r->opts.precision == OIM_PREC_AUTO) prec = OIM_PREC_FP32;
    }
    r->form = form;
    r->prec = prec;
    // the 16-bit stream form moves octets of replicas with 32-byte accesses
    if (form == OIM_FORM_STREAM && prec != OIM_PREC_FP32) r->R_pad = (r->R + 7) & ~7;
    if (form == OIM_FORM_RESIDENT) {
        cudaError_t e = plan_resident(*r->p, r->R_pad, prec, r->opts.replicas_per_block,
                                      r->opts.threads_per_block, &r->plan);
        if (e != cudaSuccess)
            return fail(OIM_EUNSUPPORTED,
                        "resident form: one replica of the largest graph does not fit in "
                        "shared memory, or the requested replicas per block is invalid");
    }
    return OIM_OK;
}

int allocate_run(oim_run_s* r) {
    const size_t state = (size_t)r->p->nodes * r->R_pad;
    const int G = r->p->G;
    OIM_CUDA(dev_alloc(&r->d_theta[0], state), "cudaMalloc(theta)");
    OIM_CUDA(dev_alloc(&r->d_spins, state), "cudaMalloc(spins)");
    OIM_CUDA(dev_alloc(&r->d_score, (size_t)G * r->R_pad), "cudaMalloc(score)");
    OIM_CUDA(dev_alloc(&r->d_energy, (size_t)G * r->R_pad), "cudaMalloc(energy)");
    OIM_CUDA(dev_alloc(&r->d_err, 1), "cudaMalloc(err)");
    OIM_CUDA(dev_alloc(&r->d_seed, 1), "cudaMalloc(seed)");
    OIM_CUDA(dev_alloc(&r->d_t0, 1), "cudaMalloc(t0)");
    if (r->form == OIM_FORM_PERSISTENT) OIM_CUDA(dev_alloc(&r->d_bar, 2), "cudaMalloc(grid barrier)");
    if (r->form == OIM_FORM_STREAM || r->form == OIM_FORM_MIXED || r->form == OIM_FORM_PERSISTENT) {
        // a step reads and writes only its own node's phases, so they are updated in
        // place (one buffer under both parities); only the (cos, sin) cache, which the
        // neighbours read, needs the second buffer
        r->d_theta[1] = r->d_theta[0];
        // (cos, sin) pairs: float2, or two 16-bit values in the FP16 / BF16 variant
        const size_t pair = r->prec == OIM_PREC_FP32 ? sizeof(float2) : sizeof(uint32_t);
        OIM_CUDA(cudaMalloc(&r->d_cs[0], state * pair), "cudaMalloc(cs)");
        OIM_CUDA(cudaMalloc(&r->d_cs[1], state * pair), "cudaMalloc(cs)");
    }
    if (r->form == OIM_FORM_GEMM) {
        int rc = gemm_setup(*r, 0);
        if (rc != OIM_OK) return rc;
    }
    if (r->form == OIM_FORM_MIXED) {
        std::vector<char> csr_member((size_t)r->p->G, 0);
        for (int g = 0; g < r->p->G; ++g) {
            if (r->graph_forms[(size_t)g] == OIM_FORM_GEMM) {
                int rc = gemm_setup(*r, g);
                if (rc != OIM_OK) return rc;
            } else {
                csr_member[(size_t)g] = 1;
            }
        }
        // the step kernels of the CSR members take only their slots
        StreamSlots sl = build_stream_slots(r->p, csr_member);
        OIM_CUDA(dev_alloc(&r->d_srow_sub, sl.srow.size()), "cudaMalloc(member rows)");
        OIM_CUDA(dev_alloc(&r->d_shead_sub, sl.shead.size()), "cudaMalloc(member row heads)");
        OIM_CUDA(dev_alloc(&r->d_sdesc_sub, sl.sdesc.size()), "cudaMalloc(member slot descriptors)");
        OIM_CUDA(upload_stream_slots(sl, r->d_srow_sub, r->d_shead_sub, r->d_sdesc_sub), "upload member slots");
        r->sub_slots = (int32_t)sl.srow.size();
        if (r->sub_slots > 0 && !r->gemms.empty()) {
            OIM_CUDA(cudaStreamCreateWithFlags(&r->aux, cudaStreamNonBlocking), "create dense-member stream");
            OIM_CUDA(cudaEventCreateWithFlags(&r->ev_fork, cudaEventDisableTiming), "create fork event");
            OIM_CUDA(cudaEventCreateWithFlags(&r->ev_join, cudaEventDisableTiming), "create join event");
        }
    }
    if (r->form == OIM_FORM_STREAM && r->readout_every > 0) {
        OIM_CUDA(cudaStreamCreateWithFlags(&r->aux_score, cudaStreamNonBlocking), "create score stream");
        OIM_CUDA(cudaEventCreateWithFlags(&r->ev_spins, cudaEventDisableTiming), "create spins event");
        OIM_CUDA(cudaEventCreateWithFlags(&r->ev_scored, cudaEventDisableTiming), "create score event");
    }
    // graphs scored on the tensor cores leave the CSR score pass
    r->score_ranges.clear();
    r->score_split = false;
    if (!r->opts.csr_scores) {
        std::vector<int2> tc;
        for (const GemmState& st : r->gemms)
            if (st.score_tc) {
                const GraphDev& gd = r->p->graphs[(size_t)st.graph];
                tc.push_back(make_int2(gd.node_off, gd.node_off + gd.n));
            }
        std::sort(tc.begin(), tc.end(), [](int2 a, int2 b) { return a.x < b.x; });
        int lo = 0;
        for (const int2& c : tc) {
            if (c.x > lo) r->score_ranges.push_back(make_int2(lo, c.x));
            lo = c.y;
        }
        if (lo < r->p->nodes) r->score_ranges.push_back(make_int2(lo, (int)r->p->nodes));
        r->score_split = !tc.empty();
    }
    if (r->form == OIM_FORM_RESIDENT) {
        const auto& items = r->plan.items;
        OIM_CUDA(dev_alloc(&r->d_items, items.size()), "cudaMalloc(items)");
        OIM_CUDA(cudaMemcpy(r->d_items, items.data(), items.size() * sizeof(int4),
                            cudaMemcpyHostToDevice),
                 "upload items");
    }
    OIM_CUDA(cudaMemset(r->d_err, 0, sizeof(int32_t)), "cudaMemset(err)");
    return OIM_OK;
}

// The step base of a replayed chunk of steps moves on by the chunk's length.
__global__ void advance_t0_kernel(int32_t* d_t0, int32_t steps) { *d_t0 += steps; }

cudaError_t launch_advance_t0(int32_t* d_t0, int32_t steps, cudaStream_t s) {
    advance_t0_kernel<<<1, 1, 0, s>>>(d_t0, steps);
    return cudaGetLastError();
}

// Steps per replay of a captured chunk: the readout period (so each chunk ends on a
// readout), doubled until it is even (the buffer parity follows the step index) and at
// least 32 steps; 0 where chunks do not apply (checkpointed runs, runs shorter than a
// chunk).
int64_t step_chunk_length(const oim_run_s& r) {
    if ((r.form != OIM_FORM_STREAM && r.form != OIM_FORM_GEMM && r.form != OIM_FORM_MIXED) || r.ckpt_every > 0)
        return 0;
    int64_t L = r.readout_every > 0 ? r.readout_every : 64;
    while ((L & 1) || L < 32) L *= 2;
    return (L <= r.steps && L <= (1 << 20)) ? L : 0;
}

// The per-step forms' work, part by part: the CSR step kernel over the stream form's
// nodes (every graph of the stream form, the CSR members of a mixed run) and the
// tensor-core step of each dense graph (the dense form's one graph, the dense members).
bool has_csr_part(const oim_run_s& r) {
    return r.form == OIM_FORM_STREAM || (r.form == OIM_FORM_MIXED && r.sub_slots > 0);
}

cudaError_t init_parts(const oim_run_s& r, cudaStream_t s) {
    cudaError_t e = has_csr_part(r) ? launch_init_stream(r, s) : cudaSuccess;
    for (size_t k = 0; k < r.gemms.size() && e == cudaSuccess; ++k) e = launch_gemm_init(r, (int)k, s);
    return e;
}

cudaError_t step_parts(const oim_run_s& r, int64_t t, const int32_t* d_t0, cudaStream_t s) {
    cudaError_t e = has_csr_part(r) ? launch_step_stream(r, t, d_t0, s) : cudaSuccess;
    for (size_t k = 0; k < r.gemms.size() && e == cudaSuccess; ++k)
        e = launch_gemm_step_at(r, (int)k, t, d_t0, s);
    return e;
}

// the dense graphs' phases into the common layout (readouts and the end of a run); at
// readouts (scored_only) only those of the graphs that the CSR score pass scores
cudaError_t common_parts(const oim_run_s& r, cudaStream_t s, bool scored_only = false) {
    cudaError_t e = cudaSuccess;
    for (size_t k = 0; k < r.gemms.size() && e == cudaSuccess; ++k)
        if (!(scored_only && tc_scored(r, (int)k))) e = launch_gemm_to_common(r, (int)k, r.d_theta[0], s);
    return e;
}

// The readout after `b` steps (an offset from *d_t0 in a replayed chunk) into slot
// `slot`: the graphs scored on the tensor cores from their spins in the X^T buffer that
// step b - 1 read (the next step writes it again), the others by the CSR score pass.
cudaError_t score_parts(const oim_run_s& r, const float* th, int64_t slot, const int32_t* d_t0, int64_t b,
                        cudaStream_t s) {
    cudaError_t e = cudaSuccess;
    for (size_t k = 0; k < r.gemms.size() && e == cudaSuccess; ++k)
        if (tc_scored(r, (int)k))
            e = launch_gemm_score(r, (int)k, slot, d_t0, (int32_t)b, (int)((b - 1) & 1), s);
    if (e == cudaSuccess && !(r.score_split && r.score_ranges.empty()))
        e = d_t0 ? launch_score_at(r, th, 0, d_t0, (int32_t)b, s) : launch_score(r, th, slot, s);
    return e;
}

// The phases in the common layout after step t (the stream form alternates buffer
// parity with the step; its two buffers alias, and the other forms keep one).
float* readout_theta(const oim_run_s& r, int64_t t) {
    return r.form == OIM_FORM_STREAM ? r.d_theta[(t + 1) & 1] : r.d_theta[0];
}

// The persistent form: init, then the steps between two readouts in one cooperative
// launch each, a score pass after each readout step (launched directly: a run is a few
// launches per readout period).
int enqueue_persistent(oim_run_s* r) {
    cudaStream_t s = r->stream;
    cudaError_t e = cudaMemsetAsync(r->d_bar, 0, 2 * sizeof(unsigned), s);
    if (e == cudaSuccess) e = launch_init_stream(*r, s);
    const int64_t re = r->readout_every;
    for (int64_t a = 0; a < r->steps && e == cudaSuccess;) {
        const int64_t b = re > 0 ? std::min<int64_t>(r->steps, (a / re + 1) * re) : r->steps;
        e = launch_persistent_steps(*r, a, b, s);
        if (e == cudaSuccess && re > 0 && b % re == 0) e = launch_score(*r, r->d_theta[0], b / re - 1, s);
        a = b;
    }
    if (e != cudaSuccess) return cuda_fail(e, "persistent-form launch");
    return OIM_OK;
}

// Steps [t0, t1) (offsets from *d_t0 in a replayed chunk, which starts on a readout
// boundary; the steps themselves otherwise) with a score pass after every readout step
// (dense graphs first copy their phases to the common layout).  The graphs of a batch
// never read one another's state, so a mixed run's two parts need to meet only at the
// readouts: between them the dense members step on the run's second stream, forked
// from q and joined back before the readout.
cudaError_t enqueue_steps(const oim_run_s& r, int64_t t0, int64_t t1, const int32_t* d_t0, cudaStream_t q) {
    cudaError_t e = cudaSuccess;
    bool scoring = false;   // a readout's scoring is running on the score stream
    const bool fork = r.aux != nullptr;
    for (int64_t a = t0; a < t1 && e == cudaSuccess;) {
        const int64_t re = r.readout_every;
        const int64_t b = re > 0 ? std::min<int64_t>(t1, (a / re + 1) * re) : t1;
        if (fork) {
            e = cudaEventRecord(r.ev_fork, q);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(r.aux, r.ev_fork, 0);
            for (int64_t t = a; t < b && e == cudaSuccess; ++t) e = launch_step_stream(r, t, d_t0, q);
            for (int64_t t = a; t < b && e == cudaSuccess; ++t)
                for (size_t k = 0; k < r.gemms.size() && e == cudaSuccess; ++k)
                    e = launch_gemm_step_at(r, (int)k, t, d_t0, r.aux);
            if (e == cudaSuccess) e = cudaEventRecord(r.ev_join, r.aux);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(q, r.ev_join, 0);
        } else {
            for (int64_t t = a; t < b && e == cudaSuccess; ++t) e = step_parts(r, t, d_t0, q);
        }
        if (e == cudaSuccess && re > 0 && b % re == 0) {
            float* th = readout_theta(r, b - 1);
            if (r.aux_score) {
                // the spins on the run's stream (once the previous readout's scoring has
                // read its spins), their scoring on the second stream beside the next steps
                if (scoring) e = cudaStreamWaitEvent(q, r.ev_scored, 0);
                if (e == cudaSuccess) e = launch_spins(r, th, q);
                if (e == cudaSuccess) e = cudaEventRecord(r.ev_spins, q);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(r.aux_score, r.ev_spins, 0);
                if (e == cudaSuccess) e = launch_score_pass(r, b / re - 1, d_t0, (int32_t)b, r.aux_score);
                if (e == cudaSuccess) e = cudaEventRecord(r.ev_scored, r.aux_score);
                scoring = true;
            } else {
                e = common_parts(r, q, true);
                if (e == cudaSuccess) e = score_parts(r, th, b / re - 1, d_t0, b, q);
            }
        }
        a = b;
    }
    // every scoring forked above is joined back before the steps' caller goes on
    if (e == cudaSuccess && scoring) e = cudaStreamWaitEvent(q, r.ev_scored, 0);
    return e;
}

// A per-step form as init, steps / L replays of one captured chunk of L steps and its
// score passes (steps and readout slots read from the device step base, which the
// chunk's last node moves on by L), and the remaining steps launched directly.  The
// chunk is captured once per (L, dt, readout period) and kept with the run.  When it has
// to be captured, the first L steps are launched directly before the capture, so that
// the GPU runs them while the host records and instantiates the chunk.
int enqueue_stream_chunks(oim_run_s* r, int64_t L) {
    cudaStream_t s = r->stream;
    cudaError_t e = init_parts(*r, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(r->d_t0, 0, sizeof(int32_t), s);
    if (e != cudaSuccess) return cuda_fail(e, "stream-form launch");
    int64_t first = 0;   // chunks already launched directly
    if (!r->step_chunk_exec || r->step_chunk_len != L || r->step_chunk_dt != r->dt ||
        r->step_chunk_every != r->readout_every) {
        e = enqueue_steps(*r, 0, L, nullptr, s);
        if (e == cudaSuccess) e = launch_advance_t0(r->d_t0, (int32_t)L, s);
        if (e != cudaSuccess) return cuda_fail(e, "stream-form launch");
        first = 1;
        if (r->step_chunk_exec) cudaGraphExecDestroy(r->step_chunk_exec);
        r->step_chunk_exec = nullptr;
        cudaStream_t cap = nullptr;
        OIM_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "create capture stream");
        cudaGraph_t graph = nullptr;
        e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            e = enqueue_steps(*r, 0, L, r->d_t0, cap);
            if (e == cudaSuccess) e = launch_advance_t0(r->d_t0, (int32_t)L, cap);
            cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
            if (e == cudaSuccess) e = e2;
        }
        cudaStreamDestroy(cap);
        if (e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return cuda_fail(e, "capture step chunk");
        }
        e = cudaGraphInstantiate(&r->step_chunk_exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(e, "instantiate step chunk");
        r->step_chunk_len = L;
        r->step_chunk_dt = r->dt;
        r->step_chunk_every = r->readout_every;
    }
    const int64_t chunks = r->steps / L;
    for (int64_t c = first; c < chunks; ++c) OIM_CUDA(cudaGraphLaunch(r->step_chunk_exec, s), "chunk launch");
    if (e == cudaSuccess) e = enqueue_steps(*r, chunks * L, r->steps, nullptr, s);
    if (e == cudaSuccess) e = common_parts(*r, s);
    if (e != cudaSuccess) return cuda_fail(e, "stream-form launch");
    return OIM_OK;
}

// Queue a per-step form: init, then every step, with a score pass after each readout
// step.  When capture is on, the whole sequence is recorded once into a CUDA graph
// (kernel arguments baked in) and replayed on later identical runs.
int enqueue_stream_form(oim_run_s* r) {
    const size_t state_bytes = (size_t)r->p->nodes * r->R_pad * sizeof(float);
    auto body = [&](cudaStream_t s) -> cudaError_t {
        cudaError_t e = init_parts(*r, s);
        if (r->ckpt_every <= 0) {
            if (e == cudaSuccess) e = enqueue_steps(*r, 0, r->steps, nullptr, s);
        } else if (r->d_ab) {
            // the whole trajectory: each step reads its phases from slot t and writes slot
            // t + 1 of the checkpoints, and keeps its coupling sums
            const size_t st = (size_t)r->p->nodes * r->R_pad;
            float* ck = r->d_ckpt;
            float2* cs0 = reinterpret_cast<float2*>(r->d_cs[0]);
            float2* cs1 = reinterpret_cast<float2*>(r->d_cs[1]);
            if (e == cudaSuccess) e = cudaMemcpyAsync(ck, r->d_theta[0], state_bytes, cudaMemcpyDeviceToDevice, s);
            const int64_t re = r->readout_every;
            for (int64_t t = 0; t < r->steps && e == cudaSuccess; ++t) {
                e = launch_step_stream_buffers(*r, t, ck + (size_t)t * st, (t & 1) ? cs1 : cs0,
                                               ck + (size_t)(t + 1) * st, (t & 1) ? cs0 : cs1,
                                               r->d_ab + (size_t)t * st, s);
                if (e == cudaSuccess && re > 0 && (t + 1) % re == 0)
                    e = launch_score(*r, ck + (size_t)(t + 1) * st, (t + 1) / re - 1, s);
            }
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(r->d_theta[0], ck + (size_t)r->steps * st, state_bytes,
                                    cudaMemcpyDeviceToDevice, s);
        } else {
            // checkpoints (the FP32 stream form): the phases after every ckpt_every steps
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(r->d_ckpt, r->d_theta[0], state_bytes, cudaMemcpyDeviceToDevice, s);
            for (int64_t t = 0; t < r->steps && e == cudaSuccess; ++t) {
                e = enqueue_steps(*r, t, t + 1, nullptr, s);
                if (e == cudaSuccess && (t + 1) % r->ckpt_every == 0)
                    e = cudaMemcpyAsync(r->d_ckpt + (size_t)((t + 1) / r->ckpt_every) * r->p->nodes * r->R_pad,
                                        readout_theta(*r, t), state_bytes, cudaMemcpyDeviceToDevice, s);
            }
        }
        if (e == cudaSuccess) e = common_parts(*r, s);
        return e;
    };
    if (!r->opts.use_graph) {
        cudaError_t e = body(r->stream);
        if (e != cudaSuccess) return cuda_fail(e, "stream-form launch");
        return OIM_OK;
    }
    // the seed is read from device memory, so one graph serves every seed
    const bool same = r->chunk_exec && r->graph_steps == r->steps && r->graph_dt == r->dt;
    if (!same && (r->seen_steps != r->steps || r->seen_dt != r->dt)) {
        // first execution of this shape: capturing and instantiating thousands of nodes
        // would cost more than it saves for a run made once, so the run replays a short
        // captured chunk of steps (its step base in device memory; checkpointed runs
        // launch directly); the whole run is captured if the shape comes back
        r->seen_steps = r->steps;
        r->seen_dt = r->dt;
        const int64_t L = step_chunk_length(*r);
        if (L > 0) return enqueue_stream_chunks(r, L);
        cudaError_t e = body(r->stream);
        if (e != cudaSuccess) return cuda_fail(e, "stream-form launch");
        return OIM_OK;
    }
    if (!same) {
        if (r->chunk_exec) cudaGraphExecDestroy(r->chunk_exec);
        r->chunk_exec = nullptr;
        // record on a private stream (the caller's may be the legacy default stream,
        // which cannot be captured); the graph is then launched on the caller's stream
        cudaStream_t cap = nullptr;
        OIM_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "create capture stream");
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            e = body(cap);
            cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
            if (e == cudaSuccess) e = e2;
        }
        cudaStreamDestroy(cap);
        if (e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return cuda_fail(e, "capture stream form");
        }
        e = cudaGraphInstantiate(&r->chunk_exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(e, "instantiate graph");
        r->graph_steps = r->steps;
        r->graph_dt = r->dt;
    }
    OIM_CUDA(cudaGraphLaunch(r->chunk_exec, r->stream), "graph launch");
    return OIM_OK;
}

int execute(oim_run_s* r, const float* K, const float* Ks, const float* Kn) {
    const int G = r->p->G;
    cudaStream_t s = r->stream;
    const size_t row = (size_t)G * r->steps;
    // schedules are [G][steps] per array; the device copy keeps the stride steps_cap
    for (int a = 0; a < 3; ++a) {
        const float* src = a == 0 ? K : (a == 1 ? Ks : Kn);
        if (r->steps == 0) break;
        float* dst = r->d_sched + (size_t)a * G * r->steps_cap;
        if (r->steps_cap == r->steps) {
            OIM_CUDA(cudaMemcpyAsync(dst, src, row * sizeof(float), cudaMemcpyDefault, s),
                     "copy schedule");
        } else {
            OIM_CUDA(cudaMemcpy2DAsync(dst, r->steps_cap * sizeof(float), src,
                                       r->steps * sizeof(float), r->steps * sizeof(float), G,
                                       cudaMemcpyDefault, s),
                     "copy schedule");
        }
    }
    OIM_CUDA(cudaMemsetAsync(r->d_trace, 0, (size_t)G * r->readouts_cap * r->R_pad * sizeof(double), s),
             "clear trace");
    // the per-step forms read the seed from device memory (their captured graphs are
    // replayed for any seed)
    if (r->form != OIM_FORM_RESIDENT) OIM_CUDA(launch_set_seed(r->d_seed, r->seed, s), "store seed");
    if (r->form == OIM_FORM_RESIDENT) {
        cudaError_t e = launch_resident_impl(*r, r->d_items, s);
        if (e != cudaSuccess) return cuda_fail(e, "resident launch");
        r->final_buf = 0;
    } else if (r->form == OIM_FORM_PERSISTENT) {
        int rc = enqueue_persistent(r);
        if (rc != OIM_OK) return rc;
        r->final_buf = 0;
    } else {
        int rc = enqueue_stream_form(r);
        if (rc != OIM_OK) return rc;
        r->final_buf = r->form == OIM_FORM_GEMM ? 0 : (int)(r->steps & 1);
    }
    r->ran = true;
    return OIM_OK;
}

// Makes p's device current until `scope` ends (the caller's device is restored then).
int set_device_of(const oim_problem_s* p, DeviceScope& scope) {
    OIM_CUDA(scope.enter(p->device), "cudaSetDevice");
    return OIM_OK;
}

// Checked builds: OIM_EINDEX (and the word cleared) when a kernel recorded a column
// index outside its row's graph since the last check; other builds never record one.
int take_check_word(oim_problem_s* p) {
#ifdef OIM_CHECKS
    if (!p || !p->d_check) return OIM_OK;
    int32_t w = 0;
    OIM_CUDA(cudaMemcpy(&w, p->d_check, sizeof(w), cudaMemcpyDeviceToHost), "read check word");
    if (w != 0) {
        OIM_CUDA(cudaMemset(p->d_check, 0, sizeof(w)), "clear check word");
        return fail(OIM_EINDEX, "a column index outside its row's graph was skipped (checked build)");
    }
#else
    (void)p;
#endif
    return OIM_OK;
}

}  // namespace

extern "C" {

void oim_default_opts(oim_run_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->form = OIM_FORM_AUTO;
    o->precision = OIM_PREC_AUTO;
    o->readout_every = 0;
    o->stream = nullptr;
    o->use_graph = 1;
}

const char* oim_version(void) { return "liboim 0.1 (sm_103a)"; }

const char* oim_last_error(void) { return g_last_error.c_str(); }

int oim_create_problem(int32_t n, int32_t q, int64_t nnz, const int64_t* row_ptr,
                       const int32_t* col_idx, const float* weights, uint32_t flags,
                       oim_problem_t* out) {
    g_last_error.clear();
    if (!out) return fail(OIM_EINVAL, "out is NULL");
    *out = nullptr;
    if (n < 1 || n >= (1 << 30)) return fail(OIM_EINVAL, "n out of range");
    if (q < 2 || q > 16) return fail(OIM_EINVAL, "q must be in [2, 16]");
    if (nnz < 0 || nnz >= ((int64_t)1 << 31)) return fail(OIM_EINVAL, "nnz out of range");
    if (!row_ptr || (nnz > 0 && !col_idx)) return fail(OIM_EINVAL, "NULL CSR array");
    // host arrays are read in place; device arrays are copied to the host first
    std::vector<int64_t> rp_store;
    std::vector<int32_t> ci_store;
    std::vector<float> w_store;
    const int64_t* rp = nullptr;
    const int32_t* ci = nullptr;
    const float* w = nullptr;
    OIM_CUDA(view(rp, rp_store, row_ptr, (size_t)n + 1), "read row_ptr");
    OIM_CUDA(view(ci, ci_store, col_idx, (size_t)nnz), "read col_idx");
    if (weights) {
        OIM_CUDA(view(w, w_store, weights, (size_t)nnz), "read weights");
    } else {
        w_store.assign((size_t)nnz, 1.0f);
        w = w_store.data();
    }
    if (rp[0] != 0 || rp[n] != nnz) return fail(OIM_EINVAL, "row_ptr[0] must be 0 and row_ptr[n] = nnz");
    // one pass: the structure checks, the longest row, the weight of the upper triangle
    // (summed in row order) and whether every weight is +-1 / an integer
    int32_t max_deg = 0;
    double wt = 0.0;
    bool unit = true, integer = true;
    for (int32_t i = 0; i < n; ++i) {
        if (rp[i + 1] < rp[i]) return fail(OIM_EINVAL, "row_ptr must be nondecreasing");
        max_deg = std::max<int32_t>(max_deg, (int32_t)(rp[i + 1] - rp[i]));
        int32_t prev = -1;
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
            const int32_t j = ci[e];
            const float x = w[e];
            if (j < 0 || j >= n) return fail(OIM_EINVAL, "column index out of range");
            if (j == i) return fail(OIM_EINVAL, "diagonal entry (self coupling) in row " + std::to_string(i));
            if (j <= prev) return fail(OIM_EINVAL, "columns must increase within a row");
            if (!std::isfinite(x)) return fail(OIM_EINVAL, "non-finite weight");
            prev = j;
            if (j > i) wt += (double)x;
            unit &= std::fabs(x) == 1.0f;
            integer &= x == std::floor(x);
        }
    }
    if (!(flags & OIM_FLAG_SKIP_SYMMETRY_CHECK)) {
        // Rows are visited in increasing order, so for each row j the entries (j, i) that
        // mirror the visited (i, j) come in increasing i, that is in row j's column
        // order: one cursor per row walks them, and every cursor must end at its row's
        // end (each entry matched exactly once, with the same weight).
        std::vector<int64_t> cur(rp, rp + n);
        for (int32_t i = 0; i < n; ++i)
            for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
                const int32_t j = ci[e];
                const int64_t f = cur[j];
                if (f >= rp[j + 1] || ci[f] != i || w[f] != w[e])
                    return fail(OIM_EINVAL, "coupling matrix is not symmetric at (" + std::to_string(i) +
                                                ", " + std::to_string(j) + ")");
                cur[j] = f + 1;
            }
        for (int32_t j = 0; j < n; ++j)
            if (cur[j] != rp[j + 1])
                return fail(OIM_EINVAL, "coupling matrix is not symmetric: entry (" + std::to_string(j) +
                                            ", " + std::to_string(ci[cur[j]]) + ") has no mirror");
    }
    oim_problem_s* p = new (std::nothrow) oim_problem_s();
    if (!p) return fail(OIM_ENOMEM, "host allocation");
    cudaGetDevice(&p->device);
    p->q = q;
    p->G = 1;
    p->nodes = n;
    p->nnz = nnz;
    p->max_n = n;
    GraphDev gd{};
    gd.n = n;
    gd.node_off = 0;
    gd.edge_off = 0;
    gd.max_deg = max_deg;
    gd.wtot = wt;
    p->graphs.push_back(gd);
    p->h_rowp.resize((size_t)n + 1);
    for (int32_t i = 0; i <= n; ++i) p->h_rowp[i] = (int32_t)rp[i];
    p->unit_weights = unit;
    p->integer_weights = integer;
    // With +-1 weights each row is stored positive entries first (each part in
    // ascending column order), so the coupling gather is two sign-free loops; h_col
    // carries the sign in its top bit.  (Each entry's place is computed, not branched
    // on: the signs of a +-1 graph are random.)
    p->h_col_plain.resize((size_t)nnz);
    p->h_col.resize((size_t)nnz);
    p->h_w.resize((size_t)nnz);
    p->h_split.resize((size_t)n);
    for (int32_t i = 0; i < n; ++i) {
        const int64_t b = rp[i], en = rp[i + 1];
        if (!unit) {
            std::copy(ci + b, ci + en, p->h_col_plain.begin() + b);
            std::copy(w + b, w + en, p->h_w.begin() + b);
            for (int64_t e = b; e < en; ++e) p->h_col[e] = (uint32_t)ci[e];
            p->h_split[i] = (int32_t)en;
            continue;
        }
        int64_t nneg = 0;
        for (int64_t e = b; e < en; ++e) nneg += w[e] < 0.f;
        int64_t pos = b, neg = en - nneg;
        p->h_split[i] = (int32_t)neg;
        for (int64_t e = b; e < en; ++e) {
            const bool ng = w[e] < 0.f;
            const int64_t at = ng ? neg : pos;
            p->h_col_plain[at] = ci[e];
            p->h_col[at] = (uint32_t)ci[e] | (ng ? kSignBit : 0u);
            p->h_w[at] = w[e];
            neg += ng;
            pos += !ng;
        }
    }
    p->h_order.resize((size_t)n);
    for (int32_t i = 0; i < n; ++i) p->h_order[i] = i;
    std::stable_sort(p->h_order.begin(), p->h_order.end(), [&](int32_t a, int32_t b) {
        return rp[a + 1] - rp[a] > rp[b + 1] - rp[b];
    });
    if (!(flags & OIM_FLAG_DEFER_UPLOAD)) {
        int rc = upload_problem(p);
        if (rc != OIM_OK) {
            free_problem(p);
            delete p;
            return rc;
        }
    }
    *out = p;
    return OIM_OK;
}

namespace {

// oim_create_batch, with the upload left to the first run when `defer` is set.  The
// members' rows are copied into the batch graph by graph on host threads.
int create_batch(int32_t count, const oim_problem_t* problems, bool defer, oim_problem_t* out) {
    if (!out) return fail(OIM_EINVAL, "out is NULL");
    *out = nullptr;
    if (count < 1 || !problems) return fail(OIM_EINVAL, "count must be >= 1");
    for (int32_t k = 0; k < count; ++k) {
        if (!problems[k]) return fail(OIM_EINVAL, "NULL problem in batch");
        if (problems[k]->G != 1) return fail(OIM_EINVAL, "a batch cannot contain a batch");
        if (problems[k]->q != problems[0]->q) return fail(OIM_EINVAL, "mixed q in batch");
    }
    int64_t nodes = 0, nnz = 0;
    for (int32_t k = 0; k < count; ++k) {
        nodes += problems[k]->nodes;
        nnz += problems[k]->nnz;
    }
    if (nodes >= (1 << 30) || nnz >= ((int64_t)1 << 31)) return fail(OIM_EINVAL, "batch too large");
    oim_problem_s* p = new (std::nothrow) oim_problem_s();
    if (!p) return fail(OIM_ENOMEM, "host allocation");
    cudaGetDevice(&p->device);
    p->q = problems[0]->q;
    p->G = count;
    p->nodes = nodes;
    p->nnz = nnz;
    for (int32_t k = 0; k < count; ++k) {
        p->unit_weights = p->unit_weights && problems[k]->unit_weights;
        p->integer_weights = p->integer_weights && problems[k]->integer_weights;
    }
    p->h_rowp.resize((size_t)nodes + 1);
    p->h_split.resize((size_t)nodes);
    p->h_order.resize((size_t)nodes);
    p->h_col_plain.resize((size_t)nnz);
    p->h_col.resize((size_t)nnz);
    p->h_w.resize((size_t)nnz);
    p->h_rowp[0] = 0;
    std::vector<int64_t> noffs((size_t)count), eoffs((size_t)count);
    int64_t noff = 0, eoff = 0;
    for (int32_t k = 0; k < count; ++k) {
        GraphDev gd = problems[k]->graphs[0];
        gd.node_off = (int32_t)noff;
        gd.edge_off = (int32_t)eoff;
        p->graphs.push_back(gd);
        p->max_n = std::max(p->max_n, gd.n);
        noffs[(size_t)k] = noff;
        eoffs[(size_t)k] = eoff;
        noff += gd.n;
        eoff += problems[k]->nnz;
    }
    // the member's columns moved by its node offset; the packed words keep their sign
    // bit only where the whole batch has +-1 weights
    const uint32_t keep = p->unit_weights ? kSignBit : 0u;
    parallel_for(count, nnz, [&](int64_t k) {
        const oim_problem_s* s = problems[k];
        const int64_t no = noffs[(size_t)k], eo = eoffs[(size_t)k];
        for (int32_t i = 0; i < s->graphs[0].n; ++i) {
            p->h_rowp[(size_t)(no + i + 1)] = (int32_t)(eo + s->h_rowp[i + 1]);
            p->h_split[(size_t)(no + i)] = (int32_t)(eo + s->h_split[i]);
            p->h_order[(size_t)(no + i)] = s->h_order[i];
        }
        for (int64_t e = 0; e < s->nnz; ++e) {
            const int32_t c = s->h_col_plain[(size_t)e] + (int32_t)no;
            p->h_col_plain[(size_t)(eo + e)] = c;
            p->h_col[(size_t)(eo + e)] = (uint32_t)c | (s->h_col[(size_t)e] & keep);
        }
        std::copy(s->h_w.begin(), s->h_w.end(), p->h_w.begin() + eo);
    });
    if (!defer) {
        const int rc = upload_problem(p);
        if (rc != OIM_OK) {
            free_problem(p);
            delete p;
            return rc;
        }
    }
    *out = p;
    return OIM_OK;
}

}  // namespace

int oim_create_batch(int32_t count, const oim_problem_t* problems, oim_problem_t* out) {
    g_last_error.clear();
    return create_batch(count, problems, false, out);
}

int oim_create_batch_csr(int32_t count, const int32_t* n, int32_t q, const int64_t* nnz,
                         const int64_t* const* row_ptr, const int32_t* const* col_idx,
                         const float* const* weights, uint32_t flags, oim_problem_t* out) {
    NvtxRange range("oim_create_batch_csr");
    g_last_error.clear();
    if (!out) return fail(OIM_EINVAL, "out is NULL");
    *out = nullptr;
    if (count < 1) return fail(OIM_EINVAL, "count must be >= 1");
    if (!n || !nnz || !row_ptr || !col_idx) return fail(OIM_EINVAL, "NULL per-graph array");
    // each graph as oim_create_problem would take it (kept on the host), on host threads;
    // a worker thread starts on device 0, so it is first moved to the caller's device
    int dev = 0;
    const bool have_dev = cudaGetDevice(&dev) == cudaSuccess;
    std::vector<oim_problem_t> members((size_t)count, nullptr);
    std::vector<int> rcs((size_t)count, OIM_OK);
    std::vector<std::string> msgs((size_t)count);
    int64_t work = 0;
    for (int32_t k = 0; k < count; ++k) work += std::max<int64_t>(nnz[k], 0) + std::max<int32_t>(n[k], 0);
    parallel_for(count, work, [&](int64_t k) {
        if (have_dev) cudaSetDevice(dev);
        try {
            rcs[(size_t)k] = oim_create_problem(n[k], q, nnz[k], row_ptr[k], col_idx[k],
                                                weights ? weights[k] : nullptr, flags | OIM_FLAG_DEFER_UPLOAD,
                                                &members[(size_t)k]);
            if (rcs[(size_t)k] != OIM_OK) msgs[(size_t)k] = oim_last_error();
        } catch (...) {   // a host allocation that failed on a worker thread
            rcs[(size_t)k] = OIM_ENOMEM;
            msgs[(size_t)k] = "host allocation";
        }
    });
    int rc = OIM_OK;
    for (int32_t k = 0; k < count && rc == OIM_OK; ++k)
        if (rcs[(size_t)k] != OIM_OK) rc = fail(rcs[(size_t)k], "graph " + std::to_string(k) + ": " + msgs[(size_t)k]);
    if (rc == OIM_OK) rc = create_batch(count, members.data(), (flags & OIM_FLAG_DEFER_UPLOAD) != 0, out);
    for (oim_problem_t m : members)
        if (m) {
            // never uploaded: host memory only
            free_problem(m);
            delete m;
        }
    return rc;
}

int oim_problem_info(oim_problem_t p, int32_t* graphs, int64_t* nodes, int64_t* nnz, int32_t* q) {
    if (!p) return fail(OIM_EINVAL, "NULL problem");
    if (graphs) *graphs = p->G;
    if (nodes) *nodes = p->nodes;
    if (nnz) *nnz = p->nnz;
    if (q) *q = p->q;
    return OIM_OK;
}

void oim_destroy_problem(oim_problem_t p) {
    if (!p) return;
    DeviceScope scope;
    scope.enter(p->device);
    free_problem(p);
    delete p;
}

int oim_run(oim_problem_t p, const float* K, const float* Ks, const float* Kn, float dt,
            int64_t steps, int32_t replicas, uint64_t seed, const oim_run_opts* opts,
            oim_run_t* out) {
    NvtxRange range("oim_run");
    g_last_error.clear();
    if (!out) return fail(OIM_EINVAL, "out is NULL");
    *out = nullptr;
    if (!p) return fail(OIM_EINVAL, "NULL problem");
    if (replicas < 1 || replicas > (1 << 20)) return fail(OIM_EINVAL, "replicas out of range");
    int rc = validate_schedule_args(dt, steps);
    if (rc != OIM_OK) return rc;
    if (steps > 0 && (!K || !Ks || !Kn)) return fail(OIM_EINVAL, "NULL schedule");
    oim_run_opts o;
    if (opts) o = *opts; else oim_default_opts(&o);
    if (o.readout_every < 0) return fail(OIM_EINVAL, "readout_every must be >= 0");
    DeviceScope scope;
    rc = set_device_of(p, scope);
    if (rc != OIM_OK) return rc;
    rc = ensure_uploaded(p);
    if (rc != OIM_OK) return rc;
    oim_run_s* r = new (std::nothrow) oim_run_s();
    if (!r) return fail(OIM_ENOMEM, "host allocation");
    r->p = p;
    r->opts = o;
    r->R = replicas;
    r->R_pad = (replicas + 3) & ~3;
    r->readout_every = o.readout_every;
    r->stream = static_cast<cudaStream_t>(o.stream);
    r->device = p->device;
    r->steps = steps;
    r->seed = seed;
    r->dt = dt;
    r->n_readouts = r->readout_every > 0 ? steps / r->readout_every : 0;
    r->ckpt_every = o.checkpoint_every;
    rc = choose_form(r);
    if (rc == OIM_OK) rc = allocate_run(r);
    if (rc == OIM_OK) rc = ensure_step_buffers(r, steps);
    if (rc == OIM_OK) rc = execute(r, K, Ks, Kn);
    if (rc != OIM_OK) {
        free_run_buffers(r);
        delete r;
        return rc;
    }
    *out = r;
    return OIM_OK;
}

int oim_rerun(oim_run_t r, const float* K, const float* Ks, const float* Kn, float dt, int64_t steps,
              uint64_t seed) {
    NvtxRange range("oim_rerun");
    g_last_error.clear();
    if (!r) return fail(OIM_EINVAL, "NULL run");
    int rc = validate_schedule_args(dt, steps);
    if (rc != OIM_OK) return rc;
    if (steps > 0 && (!K || !Ks || !Kn)) return fail(OIM_EINVAL, "NULL schedule");
    DeviceScope scope;
    rc = set_device_of(r->p, scope);
    if (rc != OIM_OK) return rc;
    r->steps = steps;
    r->seed = seed;
    r->dt = dt;
    r->n_readouts = r->readout_every > 0 ? steps / r->readout_every : 0;
    rc = ensure_step_buffers(r, steps);
    if (rc != OIM_OK) return rc;
    return execute(r, K, Ks, Kn);
}

int oim_run_sync(oim_run_t r) {
    if (!r) return fail(OIM_EINVAL, "NULL run");
    OIM_CUDA(cudaStreamSynchronize(r->stream), "synchronize");
    int32_t err = 0;
    OIM_CUDA(cudaMemcpy(&err, r->d_err, sizeof(err), cudaMemcpyDeviceToHost), "read error word");
    if (err != 0) return fail(OIM_ETIMEOUT, "a device-side wait gave up (error word " + std::to_string(err) + ")");
    return take_check_word(r->p);
}

int oim_run_info(oim_run_t r, int64_t* steps, int32_t* replicas, int64_t* n_readouts, int32_t* form,
                 int32_t* precision) {
    if (!r) return fail(OIM_EINVAL, "NULL run");
    if (steps) *steps = r->steps;
    if (replicas) *replicas = r->R;
    if (n_readouts) *n_readouts = r->n_readouts;
    if (form) *form = r->form;
    if (precision) *precision = r->prec;
    return OIM_OK;
}

int oim_readout(oim_run_t r, int8_t* spins, double* score, int32_t* best_replica, double* trace,
                double* energy) {
    NvtxRange range("oim_readout");
    g_last_error.clear();
    if (!r) return fail(OIM_EINVAL, "NULL run");
    if (!r->ran) return fail(OIM_ESTATE, "run has not executed");
    DeviceScope scope;
    int rc = set_device_of(r->p, scope);
    if (rc != OIM_OK) return rc;
    cudaStream_t s = r->stream;
    const int G = r->p->G;
    const float* theta = r->d_theta[r->final_buf];
    const int64_t k_final = r->readouts_cap - 1;   // spare row for the final scores
    if (score || best_replica) {
        for (int g = 0; g < G; ++g)
            OIM_CUDA(cudaMemsetAsync(r->d_trace + ((size_t)g * r->readouts_cap + k_final) * r->R_pad, 0,
                                     (size_t)r->R_pad * sizeof(double), s),
                     "clear final row");
        OIM_CUDA(score_parts(*r, theta, k_final, nullptr, r->steps, s), "score launch");
        OIM_CUDA(launch_finalize(*r, k_final, r->d_score, s), "finalize launch");
    }
    if (energy) {
        OIM_CUDA(cudaMemsetAsync(r->d_energy, 0, (size_t)G * r->R_pad * sizeof(double), s), "clear energy");
        OIM_CUDA(launch_energy_of(*r, theta, r->d_energy, s), "energy launch");
    }
    if (spins) OIM_CUDA(launch_gather(*r, theta, r->d_spins, nullptr, s), "gather launch");
    rc = oim_run_sync(r);
    if (rc != OIM_OK) return rc;
    const size_t GR = (size_t)G * r->R;
    std::vector<double> host_score;
    if (score || best_replica) {
        host_score.resize(GR);
        OIM_CUDA(cudaMemcpy(host_score.data(), r->d_score, GR * sizeof(double), cudaMemcpyDeviceToHost),
                 "read scores");
        if (score) OIM_CUDA(cudaMemcpy(score, host_score.data(), GR * sizeof(double), cudaMemcpyDefault),
                            "write scores");
        if (best_replica) {
            std::vector<int32_t> best((size_t)G);
            for (int g = 0; g < G; ++g) {
                int b = 0;
                for (int x = 1; x < r->R; ++x) {
                    const double v = host_score[(size_t)g * r->R + x], bv = host_score[(size_t)g * r->R + b];
                    if (r->p->q == 2 ? v > bv : v < bv) b = x;
                }
                best[g] = b;
            }
            OIM_CUDA(cudaMemcpy(best_replica, best.data(), G * sizeof(int32_t), cudaMemcpyDefault),
                     "write best replica");
        }
    }
    if (spins)
        OIM_CUDA(cudaMemcpy(spins, r->d_spins, (size_t)r->p->nodes * r->R, cudaMemcpyDefault), "write spins");
    if (energy) {
        std::vector<double> e((size_t)G * r->R_pad), o(GR);
        OIM_CUDA(cudaMemcpy(e.data(), r->d_energy, e.size() * sizeof(double), cudaMemcpyDeviceToHost),
                 "read energy");
        for (int g = 0; g < G; ++g)
            for (int x = 0; x < r->R; ++x) o[(size_t)g * r->R + x] = e[(size_t)g * r->R_pad + x];
        OIM_CUDA(cudaMemcpy(energy, o.data(), GR * sizeof(double), cudaMemcpyDefault), "write energy");
    }
    if (trace && r->n_readouts > 0) {
        std::vector<double> raw((size_t)G * r->readouts_cap * r->R_pad);
        OIM_CUDA(cudaMemcpy(raw.data(), r->d_trace, raw.size() * sizeof(double), cudaMemcpyDeviceToHost),
                 "read trace");
        std::vector<double> o((size_t)G * r->n_readouts * r->R);
        for (int g = 0; g < G; ++g)
            for (int64_t k = 0; k < r->n_readouts; ++k)
                for (int x = 0; x < r->R; ++x) {
                    const double a = raw[((size_t)g * r->readouts_cap + k) * r->R_pad + x];
                    o[((size_t)g * r->n_readouts + k) * r->R + x] =
                        r->p->q == 2 ? r->p->graphs[g].wtot - a : a;
                }
        OIM_CUDA(cudaMemcpy(trace, o.data(), o.size() * sizeof(double), cudaMemcpyDefault), "write trace");
    }
    return OIM_OK;
}

int oim_get_phases(oim_run_t r, float* theta) {
    g_last_error.clear();
    if (!r || !theta) return fail(OIM_EINVAL, "NULL argument");
    if (!r->ran) return fail(OIM_ESTATE, "run has not executed");
    DeviceScope scope;
    int rc = set_device_of(r->p, scope);
    if (rc != OIM_OK) return rc;
    float* tmp = nullptr;
    const size_t count = (size_t)r->p->nodes * r->R;
    OIM_CUDA(cudaMalloc(&tmp, count * sizeof(float)), "cudaMalloc(phases)");
    cudaError_t e = launch_gather(*r, r->d_theta[r->final_buf], nullptr, tmp, r->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(r->stream);
    if (e == cudaSuccess) e = cudaMemcpy(theta, tmp, count * sizeof(float), cudaMemcpyDefault);
    cudaFree(tmp);
    if (e != cudaSuccess) return cuda_fail(e, "get phases");
    return oim_run_sync(r);
}

int oim_debug_derivative(oim_problem_t p, const float* theta, int32_t replicas, float K, float Ks,
                         float* f_out) {
    g_last_error.clear();
    if (!p || !theta || !f_out) return fail(OIM_EINVAL, "NULL argument");
    if (p->G != 1) return fail(OIM_EINVAL, "debug derivative takes a single graph");
    if (replicas < 1) return fail(OIM_EINVAL, "replicas must be >= 1");
    DeviceScope scope;
    int rc = set_device_of(p, scope);
    if (rc == OIM_OK) rc = ensure_uploaded(p);
    if (rc != OIM_OK) return rc;
    const size_t count = (size_t)p->nodes * replicas;
    float *d_th = nullptr, *d_f = nullptr;
    OIM_CUDA(cudaMalloc(&d_th, count * sizeof(float)), "cudaMalloc");
    cudaError_t e = cudaMalloc(&d_f, count * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(d_th, theta, count * sizeof(float), cudaMemcpyDefault);
    if (e == cudaSuccess) e = launch_derivative(*p, d_th, replicas, K, Ks, d_f, nullptr);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(f_out, d_f, count * sizeof(float), cudaMemcpyDefault);
    cudaFree(d_th);
    if (d_f) cudaFree(d_f);
    if (e != cudaSuccess) return cuda_fail(e, "debug derivative");
    return OIM_OK;
}

int oim_debug_set_column(oim_problem_t p, int64_t entry, int32_t column, int32_t* previous) {
    g_last_error.clear();
    if (!p) return fail(OIM_EINVAL, "NULL problem");
    if (entry < 0 || entry >= p->nnz) return fail(OIM_EINVAL, "entry out of range");
    if (column < 0 || column >= p->nodes) return fail(OIM_EINVAL, "column out of range");
    {
        // the first four entries of a row are also held by the slot descriptors
        const auto it = std::upper_bound(p->h_rowp.begin(), p->h_rowp.end(), (int32_t)entry);
        const int64_t row_start = *(it - 1);
        if (entry - row_start < 4) return fail(OIM_EINVAL, "entry among the first four of its row");
    }
    DeviceScope scope;
    int rc = set_device_of(p, scope);
    if (rc == OIM_OK) rc = ensure_uploaded(p);
    if (rc != OIM_OK) return rc;
    const uint32_t packed = (uint32_t)column | (p->h_col[(size_t)entry] & kSignBit);
    const int32_t plain = column;
    if (previous) {
        uint32_t old = 0;
        OIM_CUDA(cudaMemcpy(&old, p->d_col + entry, sizeof(old), cudaMemcpyDeviceToHost), "read column");
        *previous = (int32_t)(old & ~kSignBit);
    }
    OIM_CUDA(cudaMemcpy(p->d_col + entry, &packed, sizeof(packed), cudaMemcpyHostToDevice), "write column");
    OIM_CUDA(cudaMemcpy(p->d_pcol + entry, &plain, sizeof(plain), cudaMemcpyHostToDevice), "write column");
    return OIM_OK;
}

int oim_backward(oim_run_t r, double* dK, double* dKs, double* dKn, double* loss) {
    NvtxRange range("oim_backward");
    g_last_error.clear();
    if (!r) return fail(OIM_EINVAL, "NULL run");
    if (!r->ran) return fail(OIM_ESTATE, "run has not executed");
    if (r->form != OIM_FORM_STREAM || r->prec != OIM_PREC_FP32 || r->ckpt_every <= 0 || !r->d_ckpt)
        return fail(OIM_ESTATE, "oim_backward needs a run with checkpoint_every > 0 (FP32 stream form)");
    DeviceScope scope;
    int rc = set_device_of(r->p, scope);
    if (rc != OIM_OK) return rc;
    cudaStream_t s = r->stream;
    const int G = r->p->G;
    const int64_t T = r->steps, C = r->ckpt_every;
    const size_t state = (size_t)r->p->nodes * r->R_pad;
    const int64_t seg_len = std::min<int64_t>(C, std::max<int64_t>(T, 1));
    // the whole trajectory kept by the forward pass (phases and coupling sums of every
    // step): one segment over all steps, nothing recomputed
    const bool whole = C == 1 && r->d_ab != nullptr;
    // per segment: the phases theta_t0 .. theta_t1 and the coupling sums (A, B) of its
    // steps, recomputed from the checkpoint; lambda ping-pong; two ping-pong pairs of
    // planes lambda_{t+1} (c, s)_t
    float *seg = nullptr, *lam[2] = {nullptr, nullptr}, *Y[2] = {nullptr, nullptr};
    float2 *cs[2] = {nullptr, nullptr}, *ab = nullptr;
    double *gK = nullptr, *gS = nullptr, *gN = nullptr, *gL = nullptr;
    cudaError_t e = cudaSuccess;
    auto cleanup = [&]() {
        cudaFree(seg); cudaFree(lam[0]); cudaFree(lam[1]); cudaFree(cs[0]); cudaFree(cs[1]);
        cudaFree(Y[0]); cudaFree(Y[1]); cudaFree(ab); cudaFree(gK); cudaFree(gS); cudaFree(gN); cudaFree(gL);
    };
#define OIM_BW(call, what)                     \
    do {                                       \
        e = (call);                            \
        if (e != cudaSuccess) {                \
            cleanup();                         \
            return cuda_fail(e, what);         \
        }                                      \
    } while (0)
    if (!whole) {
        OIM_BW(cudaMalloc(&seg, (size_t)(seg_len + 1) * state * sizeof(float)), "cudaMalloc(segment)");
        OIM_BW(cudaMalloc(&ab, (size_t)seg_len * state * sizeof(float2)), "cudaMalloc(coupling sums)");
    }
    OIM_BW(cudaMalloc(&lam[0], state * sizeof(float)), "cudaMalloc(lambda)");
    OIM_BW(cudaMalloc(&lam[1], state * sizeof(float)), "cudaMalloc(lambda)");
    OIM_BW(cudaMalloc(&cs[0], state * sizeof(float2)), "cudaMalloc(cs)");
    OIM_BW(cudaMalloc(&cs[1], state * sizeof(float2)), "cudaMalloc(cs)");
    OIM_BW(cudaMalloc(&Y[0], 2 * state * sizeof(float)), "cudaMalloc(planes)");
    OIM_BW(cudaMalloc(&Y[1], 2 * state * sizeof(float)), "cudaMalloc(planes)");
    const size_t gbytes = (size_t)G * std::max<int64_t>(T, 1) * sizeof(double);
    OIM_BW(cudaMalloc(&gK, gbytes), "cudaMalloc(grad)");
    OIM_BW(cudaMalloc(&gS, gbytes), "cudaMalloc(grad)");
    OIM_BW(cudaMalloc(&gN, gbytes), "cudaMalloc(grad)");
    OIM_BW(cudaMalloc(&gL, (size_t)G * sizeof(double)), "cudaMalloc(loss)");
    OIM_BW(cudaMemsetAsync(gK, 0, gbytes, s), "clear grad");
    OIM_BW(cudaMemsetAsync(gS, 0, gbytes, s), "clear grad");
    OIM_BW(cudaMemsetAsync(gN, 0, gbytes, s), "clear grad");
    OIM_BW(cudaMemsetAsync(gL, 0, (size_t)G * sizeof(double), s), "clear loss");
    // terminal adjoint and loss from the final phases
    OIM_BW(launch_adj_planes(*r, r->d_theta[r->final_buf], nullptr, Y[0], s), "adjoint planes");
    OIM_BW(launch_adj_terminal(*r, Y[0], lam[0], gL, s), "adjoint terminal");
    int cur = 0, cy = 0;
    const int64_t n_seg = whole ? 0 : (T + C - 1) / C;
    if (whole && T > 0) {
        const float* ck = r->d_ckpt;
        OIM_BW(launch_adj_planes(*r, ck + (size_t)(T - 1) * state, lam[cur], Y[cy], s), "adjoint planes");
        for (int64_t t = T - 1; t >= 0; --t) {
            const float* th = ck + (size_t)t * state;
            OIM_BW(launch_adj_step(*r, t, th, t > 0 ? th - state : nullptr, r->d_ab + (size_t)t * state, Y[cy],
                                   Y[cy ^ 1], lam[cur], lam[cur ^ 1], gK, gS, gN, s),
                   "adjoint step");
            cur ^= 1;
            cy ^= 1;
        }
    }
    for (int64_t sg = n_seg - 1; sg >= 0; --sg) {
        const int64_t t0 = sg * C, t1 = std::min<int64_t>(t0 + C, T);
        // recompute theta_t0 .. theta_t1 from the checkpoint with the forward kernel,
        // keeping the coupling sums of steps t0 .. t1 - 1
        OIM_BW(cudaMemcpyAsync(seg, r->d_ckpt + (size_t)sg * state, state * sizeof(float),
                               cudaMemcpyDeviceToDevice, s), "load checkpoint");
        OIM_BW(launch_cs_from_theta(*r, seg, cs[0], s), "recompute cache");
        for (int64_t m = 0; m < t1 - t0; ++m)
            OIM_BW(launch_step_stream_buffers(*r, t0 + m, seg + (size_t)m * state, cs[m & 1],
                                              seg + (size_t)(m + 1) * state, cs[(m + 1) & 1],
                                              ab + (size_t)m * state, s),
                   "recompute step");
        // the planes the segment's last step gathers: lambda_t1 (c, s)_{t1 - 1}
        OIM_BW(launch_adj_planes(*r, seg + (size_t)(t1 - 1 - t0) * state, lam[cur], Y[cy], s), "adjoint planes");
        for (int64_t t = t1 - 1; t >= t0; --t) {
            const float* th = seg + (size_t)(t - t0) * state;
            const float* th_prev = t > t0 ? th - state : nullptr;
            OIM_BW(launch_adj_step(*r, t, th, th_prev, ab + (size_t)(t - t0) * state, Y[cy], Y[cy ^ 1], lam[cur],
                                   lam[cur ^ 1], gK, gS, gN, s),
                   "adjoint step");
            cur ^= 1;
            cy ^= 1;
        }
    }
    OIM_BW(cudaStreamSynchronize(s), "backward");
    rc = take_check_word(r->p);
    if (rc != OIM_OK) {
        cleanup();
        return rc;
    }
    const size_t gcount = (size_t)G * T;
    if (dK && T > 0) OIM_BW(cudaMemcpy(dK, gK, gcount * sizeof(double), cudaMemcpyDefault), "write dK");
    if (dKs && T > 0) OIM_BW(cudaMemcpy(dKs, gS, gcount * sizeof(double), cudaMemcpyDefault), "write dKs");
    if (dKn && T > 0) OIM_BW(cudaMemcpy(dKn, gN, gcount * sizeof(double), cudaMemcpyDefault), "write dKn");
    if (loss) {
        std::vector<double> l((size_t)G);
        OIM_BW(cudaMemcpy(l.data(), gL, G * sizeof(double), cudaMemcpyDeviceToHost), "read loss");
        for (auto& x : l) x /= (double)r->R;
        OIM_BW(cudaMemcpy(loss, l.data(), G * sizeof(double), cudaMemcpyDefault), "write loss");
    }
#undef OIM_BW
    cleanup();
    return OIM_OK;
}

int oim_schedule_triangular(float* out, int64_t steps, float ks_max, int32_t periods) {
    if (!out && steps > 0) return fail(OIM_EINVAL, "NULL output");
    if (steps < 0 || periods < 1 || !std::isfinite(ks_max)) return fail(OIM_EINVAL, "bad waveform arguments");
    for (int64_t t = 0; t < steps; ++t) {
        const double x = (double)periods * (double)t / (double)steps;
        const double frac = x - std::floor(x);
        out[t] = (float)((double)ks_max * (1.0 - std::fabs(2.0 * frac - 1.0)));
    }
    return OIM_OK;
}

void oim_destroy_run(oim_run_t r) {
    if (!r) return;
    DeviceScope scope;
    scope.enter(r->device);
    cudaStreamSynchronize(r->stream);
    free_run_buffers(r);
    delete r;
}

}  // extern "C"
