/*
 * oim.h -- C ABI of liboim, a GB300 (sm_103a) simulator of the oscillator
 * Ising/Potts machine of "GPU-Accelerated Simulated Oscillator Ising/Potts
 * Machine Solving Combinatorial Optimization Problems" (arXiv 2505.22631).
 *
 * The library time-steps many independent replicas of the noisy Kuramoto phase
 * dynamics with sub-harmonic injection locking (Eq. 5, Algorithm 1) on one GPU,
 * reads the phases out to spins / colours (the phase threshold kernel of
 * Sec. III-B) and scores them as cuts (Ising, Eq. 1) or colouring conflicts
 * (Potts, Eq. 2).
 *
 * Conventions shared by every call:
 *  - Return value: OIM_OK (0) or a negative OIM_E* code; oim_last_error() then
 *    returns a message for the calling thread.  Outputs are written only on OIM_OK.
 *  - Pointers marked "host or device" may point to host memory (pageable or
 *    pinned) or to device memory of the current device; the library inspects
 *    them with cudaPointerGetAttributes.
 *  - Handles are owned by the library; the caller frees them with the matching
 *    oim_destroy_*.  Input arrays are copied; the caller keeps ownership.
 *  - Work is queued on the stream given in oim_run_opts (NULL = legacy default
 *    stream) and runs asynchronously; oim_readout, oim_get_phases and
 *    oim_run_sync wait for it.
 *  - Calls on one handle must not overlap from several host threads.
 *
 * Model (the readings of the paper this library implements):
 *   d theta_i = [ K_t * sum_j w_ij sin(2 pi (theta_i - theta_j))
 *                 - Ks_t * sin(2 pi q theta_i) ] dt + Kn_t * sqrt(dt) * xi_i,t
 *   theta_i <- theta_i - floor(theta_i)                      (phases in [0,1))
 * with xi ~ N(0,1) drawn from Philox4x32-10 (Salmon et al., SC'11) at counter
 * (node i, step t, replica>>2, (graph<<1)|1), key = seed, lane = replica&3,
 * Box-Muller on lane pairs (0,1),(2,3); initial phases are the uniforms
 * ((x>>9)+0.5)*2^-23 of the same generator at (i, 0, replica>>2, (graph<<1)|0).
 * Readout: spin = floor(q*theta + 1/2) mod q, taken in FP32.
 */
#ifndef OIM_H
#define OIM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define OIM_OK            0
#define OIM_EINVAL       -1   /* bad argument: size, range, malformed CSR, ...   */
#define OIM_ENOMEM       -2   /* device or host allocation failed                */
#define OIM_ECUDA        -3   /* a CUDA runtime call or kernel launch failed     */
#define OIM_ETIMEOUT     -4   /* a device-side wait gave up (error word set)     */
#define OIM_EUNSUPPORTED -5   /* valid request this build or GPU cannot serve   */
#define OIM_ESTATE       -6   /* handle in the wrong state for this call         */
#define OIM_EINDEX       -7   /* checked builds (-DOIM_CHECKS): a kernel met a    */
                              /* column index outside its row's graph and       */
                              /* skipped it (reported by oim_run_sync)          */

/* ---- integration forms ---------------------------------------------------- */
#define OIM_FORM_AUTO      0  /* chosen per graph by the autotuner               */
#define OIM_FORM_STREAM    1  /* CSR, one launch per step, state in HBM: FP32     */
                              /* cache (the plain form, AUTO) or FP16 / BF16      */
#define OIM_FORM_RESIDENT  2  /* one launch for all steps; each block keeps whole  */
                              /* replicas of one graph in shared memory           */
#define OIM_FORM_GEMM      3  /* dense coupling on the tensor cores (BF16 W x     */
                              /* [cos|sin], FP32 accumulate), one launch per step */
#define OIM_FORM_MIXED     4  /* a batch whose graphs take the form given per     */
                              /* graph in oim_run_opts.graph_forms: the CSR       */
                              /* members step together in the stream form, each   */
                              /* dense member on the tensor cores, every step     */
#define OIM_FORM_PERSISTENT 5 /* the 16-bit stream form with the steps between    */
                              /* two readouts in one cooperative launch (a grid    */
                              /* barrier per step, bounded: OIM_ETIMEOUT)          */

/* ---- storage precision of the (cos, sin) cache the coupling reads --------- */
#define OIM_PREC_AUTO 0
#define OIM_PREC_FP32 1
#define OIM_PREC_BF16 2
#define OIM_PREC_FP16 3

/* ---- problem flags -------------------------------------------------------- */
#define OIM_FLAG_SKIP_SYMMETRY_CHECK 1u  /* trust the caller that w_ij == w_ji   */
#define OIM_FLAG_DEFER_UPLOAD        2u  /* keep the graph on the host until its   */
                                         /* first run (e.g. a member of a batch)   */

typedef struct oim_problem_s* oim_problem_t;
typedef struct oim_run_s* oim_run_t;

typedef struct oim_run_opts {
    int32_t form;               /* OIM_FORM_*                                      */
    int32_t precision;          /* OIM_PREC_*                                      */
    int64_t readout_every;      /* score all replicas every this many steps (0: at */
                                /* the end only); a trace entry per readout        */
    void*   stream;             /* cudaStream_t to queue the work on               */
    int32_t use_graph;          /* per-step forms: replay a repeated run shape     */
                                /* from a CUDA graph.  Its first run replays a     */
                                /* captured chunk of steps (one readout period,    */
                                /* made even and at least 32 steps) and launches   */
                                /* the rest directly; checkpointed runs launch     */
                                /* their first run directly                        */
    int32_t replicas_per_block; /* resident form: 0 = chosen by the library        */
    int32_t threads_per_block;  /* 0 = chosen by the library; resident form: block */
                                /* size; dense form: 320 (128-wide tiles) or 576  */
                                /* (256-wide tiles)                                */
    int32_t checkpoint_every;   /* keep phases every this many steps for           */
                                /* oim_backward (0: no checkpoints; 1: every step, */
                                /* with its coupling sums when they fit)           */
    const int32_t* graph_forms; /* OIM_FORM_MIXED: int32[graphs], OIM_FORM_STREAM  */
                                /* or OIM_FORM_GEMM for each graph of the batch    */
                                /* (read by oim_run; NULL otherwise)               */
    int32_t csr_scores;         /* nonzero: every readout scores every graph with  */
                                /* the CSR pass.  0: a dense-form graph (dense     */
                                /* form, dense member of a mixed run) with q = 2   */
                                /* and integer |w_ij| <= 256 is scored on the      */
                                /* tensor cores, (sum w + s^T W s) / 4, exact      */
    int32_t reserved[5];
} oim_run_opts;

/* Fill *opts with the defaults: AUTO form and precision, readout at the end,
 * default stream, CUDA graph on, no checkpoints. */
void oim_default_opts(oim_run_opts* opts);

/* Library version string and the compute capability it was built for. */
const char* oim_version(void);

/* Message describing the last failed call on this host thread ("" if none). */
const char* oim_last_error(void);

/*
 * oim_create_problem -- upload one graph (Sec. II-C: max-cut maps each edge to
 * a coupling J_ij; colouring maps each edge to a coupling between differently
 * coloured nodes; here J_ij := w_ij, Eq. 5-6).
 *   n        number of oscillators (nodes), 1 <= n < 2^30
 *   q        number of stable phases: 2 = Ising max-cut, >= 3 = Potts colouring
 *            (the paper's N in Eq. 4-5), 2 <= q <= 16
 *   nnz      number of directed entries in the CSR (each undirected edge twice)
 *   row_ptr  int64[n+1], host or device; row_ptr[0] = 0, nondecreasing,
 *            row_ptr[n] = nnz
 *   col_idx  int32[nnz], host or device; strictly increasing within a row,
 *            0 <= col < n, no diagonal entry
 *   weights  float[nnz], host or device, finite; NULL means every weight is +1.
 *            The matrix must be symmetric (checked unless
 *            OIM_FLAG_SKIP_SYMMETRY_CHECK).
 *   out      receives the new handle.
 * Errors: OIM_EINVAL for any violation above, OIM_ENOMEM, OIM_ECUDA.
 */
int oim_create_problem(int32_t n, int32_t q, int64_t nnz, const int64_t* row_ptr,
                       const int32_t* col_idx, const float* weights, uint32_t flags,
                       oim_problem_t* out);

/*
 * oim_create_batch -- join `count` problems (same q) into one batch problem
 * whose graphs are simulated together in one launch (graph index g = position in
 * `problems`, which also selects the random stream of that graph).  The inputs
 * stay valid and owned by the caller.  Errors: OIM_EINVAL (count < 1, NULL
 * handle, mixed q, a batch inside a batch), OIM_ENOMEM, OIM_ECUDA.
 */
int oim_create_batch(int32_t count, const oim_problem_t* problems, oim_problem_t* out);

/*
 * oim_create_batch_csr -- create a batch of `count` graphs (same q) straight from
 * their CSR arrays: the same result as oim_create_problem (flags |
 * OIM_FLAG_DEFER_UPLOAD) for every graph followed by oim_create_batch and the
 * destruction of the members, with the graphs checked and laid out on up to 16
 * host threads at once (the batch's problem construction of Sec. III-C, done as
 * one call).
 *   count     number of graphs, >= 1
 *   n, nnz    int32[count], int64[count] (host): nodes and directed entries per graph
 *   q         number of stable phases, as in oim_create_problem
 *   row_ptr, col_idx   arrays of `count` pointers (host), each array host or
 *             device, each as in oim_create_problem
 *   weights   NULL (every weight +1), or `count` pointers, each NULL (that graph
 *             all +1) or float[nnz[g]] as in oim_create_problem
 *   flags     OIM_FLAG_SKIP_SYMMETRY_CHECK applies to every graph;
 *             OIM_FLAG_DEFER_UPLOAD keeps the batch on the host until its first run
 *   out       receives the batch handle; nothing of the members outlives the call
 * Errors: OIM_EINVAL (count < 1, NULL arrays, or any graph failing
 * oim_create_problem's checks: the message names the lowest-numbered such graph),
 * OIM_ENOMEM, OIM_ECUDA.
 */
int oim_create_batch_csr(int32_t count, const int32_t* n, int32_t q, const int64_t* nnz,
                         const int64_t* const* row_ptr, const int32_t* const* col_idx,
                         const float* const* weights, uint32_t flags, oim_problem_t* out);

/* Number of graphs, total nodes and total directed entries of a problem. */
int oim_problem_info(oim_problem_t p, int32_t* graphs, int64_t* nodes, int64_t* nnz, int32_t* q);

void oim_destroy_problem(oim_problem_t p);

/*
 * oim_run -- simulate `replicas` independent trajectories of every graph of p
 * for `steps` forward-Euler / Euler-Maruyama steps (Algorithm 1, Eq. 5).
 *   K, Ks, Kn  float[graphs * steps], host or device: per-step coupling
 *              strength, injection strength and noise amplitude of each graph
 *              (row g = graph g).  Algorithm 1 builds Ks as a triangular wave;
 *              any schedule is accepted.
 *   dt         step size h > 0
 *   steps      >= 0 and < 2^32
 *   replicas   1 <= replicas <= 2^20
 *   seed       key of the Philox stream
 *   opts       NULL for defaults
 *   out        receives the run handle, which owns the device state.
 * The phases start from the INIT stream.  Work is queued asynchronously.
 * Errors: OIM_EINVAL, OIM_ENOMEM, OIM_ECUDA, OIM_EUNSUPPORTED (form not
 * available for this problem, e.g. the resident form for a graph too large for
 * shared memory).
 */
int oim_run(oim_problem_t p, const float* K, const float* Ks, const float* Kn, float dt,
            int64_t steps, int32_t replicas, uint64_t seed, const oim_run_opts* opts,
            oim_run_t* out);

/*
 * oim_rerun -- simulate again with the buffers, form and options of r, from the
 * INIT stream of the new seed.  Same arguments and errors as oim_run; steps may
 * differ.  Lets a caller time or repeat runs without device allocations.
 */
int oim_rerun(oim_run_t r, const float* K, const float* Ks, const float* Kn, float dt,
              int64_t steps, uint64_t seed);

/* Wait for the run's queued work; maps a device-side error word to an error code. */
int oim_run_sync(oim_run_t r);

/*
 * oim_readout -- phase threshold (Sec. III-B: nearest stable phase k/q,
 * spin = floor(q*theta + 1/2) mod q in FP32) of the final phases, and scores.
 * Every output may be NULL; each non-NULL one is host or device memory.
 *   spins         int8[graphs][replicas][n_g] (graphs concatenated)
 *   score         double[graphs][replicas]: q == 2 the cut weight
 *                 sum_{i<j} w_ij [s_i != s_j]; q >= 3 the conflict weight
 *                 sum_{i<j} w_ij [s_i == s_j] (exact for integer weights)
 *   best_replica  int32[graphs]: replica with the largest cut (smallest
 *                 conflict weight), lowest index on ties
 *   trace         double[graphs][n_readouts][replicas]: the score of every
 *                 replica at every readout (n_readouts = steps / readout_every)
 *   energy        double[graphs][replicas]: Eq. 6 energy
 *                 sum_{i<j} w_ij cos(2 pi (theta_i - theta_j)) of the final phases
 * Synchronises the run's stream.  Errors: OIM_ESTATE, OIM_ECUDA, OIM_ETIMEOUT.
 */
int oim_readout(oim_run_t r, int8_t* spins, double* score, int32_t* best_replica,
                double* trace, double* energy);

/* Number of readouts recorded by the last run (steps / readout_every). */
int oim_run_info(oim_run_t r, int64_t* steps, int32_t* replicas, int64_t* n_readouts,
                 int32_t* form, int32_t* precision);

/*
 * oim_get_phases -- copy the final phases, float[graphs][replicas][n_g] in
 * [0,1), to host or device memory.  Synchronises.  Errors: OIM_ESTATE, OIM_ECUDA.
 */
int oim_get_phases(oim_run_t r, float* theta);

/*
 * oim_debug_set_column -- overwrite the column index of CSR entry `entry` in the
 * problem's device arrays (the host copy and the derived arrays keep the old
 * value), for testing the index checks of a checked build: with a column outside
 * the row's graph, the step, adjoint and readout kernels of a build made with
 * -DOIM_CHECKS skip the entry and oim_run_sync returns OIM_EINDEX; other builds
 * read the named node (in bounds: 0 <= column < nodes) as if it were a neighbour.
 *   entry   0 <= entry < nnz, not among the first four entries of its row (the
 *           stream form's slot descriptors also hold those)
 *   column  global node index, 0 <= column < nodes
 *   previous  host int32 (may be NULL): the entry's column before the call (rows
 *           are stored with their +1 entries first, so entry k of a row is not
 *           necessarily the caller's k-th column)
 * Synchronous.  Errors: OIM_EINVAL, OIM_ECUDA.
 */
int oim_debug_set_column(oim_problem_t p, int64_t entry, int32_t column, int32_t* previous);

/*
 * oim_debug_derivative -- the drift of Eq. 5 for given phases of one graph,
 * f_i = K sum_j w_ij sin(2 pi (theta_i - theta_j)) - Ks sin(2 pi q theta_i),
 * evaluated with the kernels' trig-cache identity in FP32.
 *   theta  float[replicas][n] (host or device), f_out float[replicas][n].
 * Synchronous.  Errors: OIM_EINVAL (batch problem), OIM_ECUDA.
 */
int oim_debug_derivative(oim_problem_t p, const float* theta, int32_t replicas, float K, float Ks,
                         float* f_out);

/*
 * oim_autotune -- pick the launch configuration of p for `replicas` replicas by
 * measurement: candidate forms (resident with a 16-bit or FP32 (cos, sin) cache,
 * several replicas-per-block and thread counts; the stream form with an FP32 or
 * FP16 cache; the dense tensor-core form for a single graph) each run
 * `probe_steps` steps twice on a
 * private stream, and the fastest is returned in *best (stream set to `stream`)
 * with its time per step in *best_us_per_step (may be NULL).  The paper leaves the
 * per-GPU batch size to the user (Sec. III-C); this chooses it, and the form,
 * per problem shape.
 *   precision_policy  OIM_PREC_AUTO (16-bit caches and BF16 allowed) or
 *                     OIM_PREC_FP32 (FP32 forms only)
 * For a batch under OIM_PREC_AUTO the mixed form is a candidate too: members that
 * look dense are probed on the tensor cores beside the others in the 16-bit stream
 * form, and when the mixed form wins, best->form is OIM_FORM_MIXED and
 * best->graph_forms points to the per-graph choice (owned by the library, valid for
 * the life of the process).
 * Decisions are cached for the process, keyed by graph sizes, nonzeros, q,
 * replicas and policy.  Synchronous.  Errors: OIM_EINVAL, OIM_EUNSUPPORTED (no
 * candidate ran), OIM_ECUDA.
 */
int oim_autotune(oim_problem_t p, int32_t replicas, int32_t precision_policy, int64_t probe_steps,
                 void* stream, oim_run_opts* best, double* best_us_per_step);

/*
 * oim_backward -- gradients of the relaxed loss L_g = (1/R) sum_r E_g(theta_T^r)
 * (Eq. 6 energy of the final phases, before thresholding) with respect to the
 * per-step schedules K_t, Ks_t, Kn_t of each graph, by the adjoint of the
 * forward-Euler map of Algorithm 1 (pattern "differentiable schedules": the
 * paper tunes K, Ks, Kn by hand, Sec. IV-B).  The noise enters pathwise: the
 * gradient is that of the trajectory with the run's own Philox draws.
 * The run must use the stream form in FP32 with checkpoint_every > 0; phases are
 * recomputed between checkpoints, so memory is checkpoint_every x state.  With
 * checkpoint_every = 1 the forward pass also keeps every step's coupling sums
 * (8 B per node-replica-step, on top of the 4 B of its phases) when they fit in
 * device memory with a tenth of it (at least 2 GiB) to spare, and the backward pass
 * then recomputes nothing; otherwise it recomputes each step from its phases.
 *   dK, dKs, dKn  double[graphs][steps] each (host or device, may be NULL)
 *   loss          double[graphs] (host or device, may be NULL): L_g
 * Synchronous.  Errors: OIM_ESTATE (no checkpoints, wrong form), OIM_ENOMEM, OIM_ECUDA.
 */
int oim_backward(oim_run_t r, double* dK, double* dKs, double* dKn, double* loss);

/*
 * oim_schedule_triangular -- Algorithm 1's injection-strength waveform (Sec. III-D:
 * Ks ramped up to Ks_max and back to zero, periodically): with
 * x = periods * t / steps, out[t] = ks_max * (1 - |2 frac(x) - 1|), t = 0..steps-1,
 * computed in double and rounded to float.  `out` is host memory.
 * Errors: OIM_EINVAL (NULL out, steps < 0, periods < 1, non-finite ks_max).
 */
int oim_schedule_triangular(float* out, int64_t steps, float ks_max, int32_t periods);

void oim_destroy_run(oim_run_t r);

/*
 * oim_debug_tc_gemm -- self-test of the tensor-core path behind the dense coupling
 * form (the matrix product W * [cos | sin] of Eq. 5's coupling sum): computes
 * D[m][n] = sum_k A[m][k] B[n][k] with tcgen05.mma, TMA-loaded 128-byte-swizzled
 * K-major BF16 operands and an FP32 TMEM accumulator.
 *   A  device bf16[M][K], B device bf16[N][K] (16-byte aligned), D device float[M][N];
 *   M and N multiples of 128, K a multiple of 64.  Synchronous.
 * Errors: OIM_EINVAL, OIM_EUNSUPPORTED (no tensor-map support in the driver),
 * OIM_ETIMEOUT (a pipeline wait gave up), OIM_ECUDA.
 */
int oim_debug_tc_gemm(const void* A, const void* B, float* D, int32_t M, int32_t N, int32_t K);

/*
 * oim_debug_tc_gemm_withhold -- the same self-test with the failure path of its
 * pipeline exercised on purpose: every mbarrier wait gives up after `wait_polls`
 * polls (instead of the library's fixed limit of about a second), and when
 * withhold_k_block >= 0 the TMA producer never loads that K block, so the MMA
 * thread's wait for it runs out.  The kernel then records the error in its error
 * word, lets the loads already in flight land, frees its TMEM and returns; the call
 * reports OIM_ETIMEOUT and the device stays usable (failure detection by a bounded
 * device wait, with no fault and no hang).  withhold_k_block = -1 withholds nothing
 * (the plain self-test with the given poll limit).  D is then partly written.
 * Errors: as oim_debug_tc_gemm; OIM_EINVAL for wait_polls < 1 or
 * withhold_k_block < -1.
 */
int oim_debug_tc_gemm_withhold(const void* A, const void* B, float* D, int32_t M, int32_t N, int32_t K,
                               int32_t withhold_k_block, uint32_t wait_polls);

/*
 * oim_score_phases_noalloc -- the cut / conflict scores of oim_readout, for
 * phases the caller supplies, computed without allocating any device memory.
 * (The paper has no counterpart: this is an interface for embedding.)
 *
 * Some callers cannot have a library call cudaMalloc or cudaFree: a server that
 * reserves all device memory up front and runs with a fixed footprint, an
 * application whose own allocator (a caching or arena allocator) owns every
 * byte of the device, or code on a latency path that cannot afford the device
 * synchronisation an allocation may cause.  This entry point uses only the
 * memory the caller passes plus a fixed scratch area that lives in the library
 * itself: OIM_NOALLOC_MAX_ACCUM doubles (1 MiB) of file-scope device memory,
 * held by every GPU that loads the library until the process exits.
 *
 *   p         problem (one graph or a batch) whose graph is on the device
 *             (not created with OIM_FLAG_DEFER_UPLOAD, or already run once)
 *   theta     device float[nodes][ld], 16-byte aligned: phase of replica r of
 *             global node v (graphs concatenated in batch order) at
 *             theta[v * ld + r], in [0,1); read in groups of four replicas
 *   replicas  1 <= replicas <= ld;  ld a multiple of 4
 *   score     device double[graphs][replicas]: as oim_readout's score (spins
 *             thresholded in FP32, cut for q == 2, conflict weight for q >= 3)
 *   stream    cudaStream_t to queue the work on (NULL = legacy default stream)
 * The work is queued asynchronously; score is valid once the stream is synchronised.
 * Errors: OIM_EINVAL (NULL or host pointers, theta not 16-byte or score not
 * 8-byte aligned, bad replicas / ld, or graphs * ld > OIM_NOALLOC_MAX_ACCUM),
 * OIM_ESTATE (graph not on the device), OIM_ECUDA.  Any node count is served
 * (the score pass strides over node chunks); the caller's current device is
 * restored before the call returns.
 * Every call shares the one scratch area and clears the part it uses before
 * use; calls whose work overlaps on the GPU (other streams, other host threads)
 * race on it and must be serialised by the caller.  The first call on a device
 * looks up the scratch area's device address (once per device, with that device
 * current); make that first call before any stream capture.
 */
#define OIM_NOALLOC_MAX_ACCUM 131072
int oim_score_phases_noalloc(oim_problem_t p, const float* theta, int32_t replicas, int32_t ld,
                             double* score, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* OIM_H */
