/*
 * apsp_fw.h - C ABI of the GB300 (sm_103a) Floyd-Warshall all-pairs shortest
 * paths library (libapspfw.so).
 *
 * Method: Costanzo et al., "Comparison of HPC Architectures for Computing
 * All-Pairs Shortest Paths. Intel Xeon Phi KNL vs NVIDIA Pascal"
 * (arXiv 2105.07298), §2.2: Floyd-Warshall (Algorithm 1) evaluated block by block
 * (the blocked FW of §2.2, "Blocked FW Algorithm": TB x TB blocks, R = N/TB
 * rounds of four dependency-ordered phases) and §3.2 (one kernel for phase 1,
 * one for phases 2+3, one for phase 4 per round).
 *
 * Common conventions
 * ------------------
 *  - Matrices are dense, row-major, with leading dimension ld >= n (elements):
 *    element (i, j) is at ptr[i * ld + j].  Columns n..ld-1 are never read or
 *    written.
 *  - Input distances = edge weights: D[i][j] is the weight of the directed
 *    edge i -> j, +INFINITY where there is no edge, 0 on the diagonal.  The
 *    library does not force the diagonal.  Negative weights are allowed as
 *    long as there is no negative cycle.  NaN gives undefined results.
 *  - Relaxation rule (Algorithm 1, read with a strict "<"): for every k,
 *    D[i][j] <- D[i][k] + D[k][j] when that sum is strictly smaller; the path
 *    matrix then records P[i][j] = k (global vertex index, int32).
 *    P[i][j] = -1 means "no intermediate vertex": the direct edge, i == j, or
 *    no path.  path(i,j) = path(i,P[i][j]) ++ path(P[i][j],j).
 *  - Device pointers are CUDA device (or managed) memory owned by the caller.
 *    The library never frees or retains them after the call returns.
 *  - stream: a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Work is enqueued asynchronously; argument errors are returned at once,
 *    before anything is enqueued; launch errors are returned as APSP_ECUDA.
 *  - Every entry point returns an apsp_status (int).
 *  - Results: on integer-valued weights every sum is exact (|D| < 2^24 in
 *    FP32, < 2^53 in FP64), so D is bit-exact with any correct algorithm.
 *    On real weights apsp_fw_f32 and apsp_fw_f64 are bit-exact (D and P) with
 *    a sequential blocked FW of the same block size (apsp_fw_block_size) in
 *    the same precision: every candidate sum is rounded once, in the
 *    paper's phase and k order.  The batched entry points compute phases 2/3
 *    as one product with the closed diagonal block instead (equal in exact
 *    arithmetic), so on real weights they are held to a relative error
 *    bound (about path length x 2^-24) rather than bit-exactness.
 */
#ifndef APSP_FW_H
#define APSP_FW_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  APSP_OK = 0,
  APSP_EINVAL = 1,        /* bad argument (null pointer, n < 0, ld < n, ...) */
  APSP_ECUDA = 2,         /* a CUDA call or launch failed */
  APSP_ENOMEM = 3,        /* device scratch allocation failed */
  APSP_EUNSUPPORTED = 4,  /* size or feature outside what the library supports */
  APSP_ETOODEEP = 5,      /* backward: a path's recursion exceeded the walk stack */
  APSP_ENEGCYCLE = 6,     /* apsp_check_negative_cycle: some D[i][i] < 0 */
  APSP_ETIMEOUT = 7       /* a kernel's bounded wait for an asynchronous copy ran out */
} apsp_status;

/* Human-readable name of a status code (static string, never NULL). */
const char *apsp_status_string(int status);

/* Library version as an integer MAJOR*10000 + MINOR*100 + PATCH. */
int apsp_version(void);

/* Block edge TB used by the single-graph kernels for a precision
 * (elem_bytes = 4 for FP32, 8 for FP64), or 0 if unsupported.  The blocked
 * schedule (and therefore the exact rounding of real-valued sums and the
 * tie-breaking of P) depends on TB. */
int apsp_fw_block_size(int elem_bytes);

/* ------------------------------------------------------------------------
 * Single graph, blocked Floyd-Warshall (§2.2 "Blocked FW Algorithm";
 * Algorithm 1 inside each block; kernels as in §3.2).
 *
 *   d_dist : n x n (leading dim ld) distances, overwritten in place:
 *            input = edge weights, output = shortest-path distances.
 *   n      : number of vertices, 0 <= n <= 262144 (n = 0 is a no-op); device
 *            memory bounds it first (D and P of FP32 take 8 n^2 bytes).
 *   ld     : leading dimension in elements, ld >= max(n, 1).
 *   d_path : optional n x n int32 path matrix with the same ld; when non-NULL
 *            it is fully written (P as described above).  May be NULL.
 *   stream : cudaStream_t as void*.  All work is ordered after earlier work
 *            on `stream`, and later work on `stream` sees the results.  With
 *            more than two blocks per side the next round's phases 1-3 run
 *            on an internal second stream (created and destroyed by the call,
 *            joined to `stream` by events), except while `stream` is being
 *            captured into a CUDA graph: then every phase runs on `stream`.
 *            Scratch (operand panels: about 32 n TB bytes for FP32, 96 n TB
 *            bytes for FP64; 128 MiB / 384 MiB at n = 32768) is stream-ordered
 *            (cudaMallocAsync / cudaFreeAsync on `stream`).
 * Returns APSP_OK, APSP_EINVAL (null d_dist with n > 0, ld < n, n > 262144),
 * APSP_ENOMEM (scratch) or APSP_ECUDA.
 * ---------------------------------------------------------------------- */
int apsp_fw_f32(float *d_dist, int64_t n, int64_t ld, int32_t *d_path, void *stream);
int apsp_fw_f64(double *d_dist, int64_t n, int64_t ld, int32_t *d_path, void *stream);

/* ------------------------------------------------------------------------
 * The same FP32 solve from and to HOST memory (the end-to-end call): copies
 * the weights to the device, runs apsp_fw_f32 there, copies D (and P) back,
 * and returns when the results are in host memory.
 *
 *   h_weights   : n x n row-major edge weights (ld = n), HOST, read only.
 *   h_dist      : n x n row-major output distances, HOST (may be h_weights).
 *   h_path      : optional n x n int32 output path matrix, HOST, or NULL.
 *   n           : 0 <= n <= 262144 (n = 0 is a no-op).
 *   d_work_dist : optional DEVICE buffer of n*n floats that the call uses as
 *                 D (a caller that solves repeatedly keeps it); NULL: one is
 *                 allocated stream-ordered on `stream` and freed before return.
 *   d_work_path : the same for P (n*n int32; used only if h_path != NULL).
 *   stream      : cudaStream_t as void*; work is ordered after earlier work on
 *                 it, and the call synchronizes it before returning.
 * Host buffers page-locked by cudaHostAlloc / cudaHostRegister copy at the
 * link's rate; pageable ones work too (the driver stages them).  The caller
 * owns every buffer.  Returns APSP_OK, APSP_EINVAL (n out of range, NULL
 * h_weights or h_dist with n > 0), APSP_ENOMEM (a work buffer), APSP_ECUDA,
 * or APSP_ETIMEOUT / APSP_EUNSUPPORTED as apsp_device_status reports them
 * (the call reads and clears those device error words).
 * ---------------------------------------------------------------------- */
int apsp_fw_f32_host(const float *h_weights, float *h_dist, int32_t *h_path, int64_t n,
                     float *d_work_dist, int32_t *d_work_path, void *stream);

/* Integer weights (int32), exact.  Same conventions with APSP_I32_INF
 * (INT32_MAX) in place of +infinity (no edge, no path).  Every int32 weight
 * is allowed (negative ones without a negative cycle).  The solve runs on the
 * FP64 path (every sum of fewer than 2^22 int32 values is exact in FP64, so D
 * is the exact integer result, bit for bit that of any correct FW) through a
 * stream-ordered n x n FP64 scratch (8 n^2 bytes).  A finite distance outside
 * [-(2^31 - 1), 2^31 - 2] is written saturated and makes the next
 * apsp_device_status return APSP_EUNSUPPORTED.  Returns as apsp_fw_f64. */
#define APSP_I32_INF 0x7fffffff
int apsp_fw_i32(int32_t *d_dist, int64_t n, int64_t ld, int32_t *d_path, void *stream);

/* ------------------------------------------------------------------------
 * Batched Floyd-Warshall (extension of the method; the paper has no batched
 * form): many independent graphs of uneven size in ONE persistent kernel
 * launch.  Graph g has n_g vertices and occupies n_g * n_g consecutive
 * elements (row-major, ld = n_g) starting at element offset off[g] of the
 * packed buffers.  Every graph is solved with the same relaxation rule as
 * above; results are bit-exact with the single-graph path on integer weights.
 * Each size class runs one of three kernel variants (apsp_batched_variant_info):
 * 64 x 64 blocks with 4 x 4 register tiles and lazy (0) or eager (1) path
 * tracking, whose phases 2/3 are one min-plus product with the closed
 * diagonal block (on real weights rounded differently from the sequential k
 * loop, within the FP32 error bound of the exact distances); or 128 x 128
 * blocks with 8 x 4 tiles (2), the single-graph phases run by one CTA, which
 * gives apsp_fw_f32's results bit for bit on any weights.  Variant 2 needs
 * per-CTA operand panels: (graph-dependent) scratch of up to
 * 2 MiB per resident CTA, held by the plan.
 *
 * Planning splits the graphs into size classes, orders them largest first
 * (longest-processing-time order) and uploads the work list.  A plan holds
 * device memory; it can be reused for any buffers with the same layout, and
 * apsp_fw_batched_run_f32 enqueues exactly one memset and one kernel launch,
 * so it can be captured in a CUDA graph.
 *
 *   h_n, h_off : HOST arrays, num_graphs entries: vertex counts (1..1024)
 *                and element offsets (each a multiple of 4, i.e. 16-byte
 *                aligned for FP32 / int32).
 *   d_dist     : packed FP32 distances, overwritten in place.
 *   d_path     : packed int32 path matrices (same offsets), or NULL.
 * apsp_fw_batched_f32 = plan + run + destroy (allocates and frees its work
 * list and panels with stream-ordered allocation on `stream`).
 * ---------------------------------------------------------------------- */
typedef struct apsp_batched_plan apsp_batched_plan;

int apsp_batched_plan_create(const int32_t *h_n, const int64_t *h_off, int32_t num_graphs,
                             apsp_batched_plan **out_plan);
int apsp_batched_plan_destroy(apsp_batched_plan *plan);
int apsp_fw_batched_run_f32(const apsp_batched_plan *plan, float *d_dist, int32_t *d_path,
                            void *stream);
int apsp_fw_batched_f32(float *d_dist, int32_t *d_path, const int32_t *h_n, const int64_t *h_off,
                        int32_t num_graphs, void *stream);

/* No-allocation form of apsp_fw_batched_f32.  The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory at
 * call time (a serving loop that forbids cudaMalloc on its hot path, code
 * whose device memory comes from an allocator CUDA does not own, or an
 * embedding where any hidden allocation is an error).  It allocates nothing:
 * no cudaMalloc/cudaFree, no stream-ordered or library allocation, no host
 * heap.  Its work list lives in one fixed device array of the library
 * (1 MiB + 16 bytes, held on every GPU that loads the library until exit),
 * so num_graphs may be at most 65536; larger batches return
 * APSP_EUNSUPPORTED before anything is enqueued.  Arguments are those of
 * apsp_fw_batched_f32 and so are the distances; the same persistent kernel
 * runs, but a size class set to variant 2 (which needs panel scratch) runs
 * variant 1 here, so path entries may break ties differently.
 *
 * Every call looks up the array's device address (cudaGetSymbolAddress, with
 * the caller's device current; this allocates nothing).  The first call on a
 * device also loads the library's module there: make that first call before
 * any stream capture on the device.  Every call shares the
 * array and it keeps the last call's contents (each call resets what must
 * start at zero); calls that overlap on the GPU (different streams or host
 * threads) race on it, so the caller must serialise them.  h_n and h_off are
 * read by asynchronous host-to-device copies on `stream`. */
int apsp_fw_batched_f32_noalloc(float *d_dist, int32_t *d_path, const int32_t *h_n,
                                const int64_t *h_off, int32_t num_graphs, void *stream);

/* Autotuner hook for the batched kernel: per size class (0..3, vertex-count
 * bounds given by apsp_batched_class_bounds) pick the variant index used by
 * later plans.  apsp_batched_num_variants reports how many variants a class
 * has; apsp_batched_variant_info gives a variant's block edge, register tile
 * (rows x columns of outputs per thread) and whether it tracks the path in
 * its inner loop (eager = 1) or recovers it after each product (0).
 * Distances are identical across variants on integer weights.  Defaults are
 * the built-in table. */
int apsp_batched_num_classes(void);
int apsp_batched_class_bounds(int cls, int32_t *lo, int32_t *hi);
int apsp_batched_num_variants(int cls);
int apsp_batched_set_variant(int cls, int variant);
int apsp_batched_get_variant(int cls);
int apsp_batched_variant_info(int variant, int32_t *block, int32_t *tile_rows, int32_t *tile_cols,
                              int32_t *eager);

/* ------------------------------------------------------------------------
 * Backward pass (extension; not in the paper).  D[i][j] is the sum of the
 * weights along path(i,j) as encoded by P, so for a loss L(D):
 *     dL/dW[u][v] = sum over (i,j) whose path uses edge (u,v) of dL/dD[i][j].
 * The kernel recomputes every path from P (nothing is stored by the forward
 * pass beyond P and D) and scatters dL/dD[i][j] onto its edges.
 *
 *   d_grad_dist : batch x (n x n, leading dim ld) upstream gradient dL/dD.
 *   d_path      : the path matrices P from the forward pass (same layout).
 *   d_dist      : the forward distances D (same layout); pairs with
 *                 D = +inf (no path) and the diagonal contribute nothing.
 *   d_grad_w    : output dL/dW (same layout), fully written: zero on the
 *                 diagonal, on non-edges and on edges no path uses.
 *   n, ld       : vertices and leading dimension (ld >= n).
 *   batch       : number of graphs, each `stride` elements after the last
 *                 (stride >= n * ld).
 *   d_status    : optional device int32; receives APSP_OK or APSP_ETOODEEP
 *                 (a path whose split recursion is deeper than 256 levels,
 *                 or a P that does not encode a path;
 *                 its contribution is then incomplete).  May be NULL.
 * Accumulation is FP32 atomic addition; the summation order is not fixed.
 * ---------------------------------------------------------------------- */
int apsp_fw_backward_f32(const float *d_grad_dist, const int32_t *d_path, const float *d_dist,
                         float *d_grad_w, int64_t n, int64_t ld, int64_t batch, int64_t stride,
                         int32_t *d_status, void *stream);

/* The same backward pass for a packed batch of uneven graphs, in the layout
 * of the batched forward: graph g has d_n[g] vertices and occupies
 * d_n[g]^2 consecutive elements (row-major, ld = d_n[g]) at element offset
 * d_off[g] of every packed buffer (gradient, P, D and the output).
 *   d_n, d_off : DEVICE arrays of num_graphs entries (int32, int64); graphs
 *                must not overlap.  A graph with d_n[g] <= 0 is skipped
 *                (d_n[g] < 0 also reports APSP_EINVAL in *d_status).
 *   d_grad_w   : fully written over every graph's region (zero on the
 *                diagonal, non-edges and unused edges); gaps between graphs
 *                are not touched.
 *   d_status   : optional device int32, as for apsp_fw_backward_f32.
 * Returns APSP_EINVAL for num_graphs < 0 or a NULL buffer with num_graphs > 0. */
int apsp_fw_backward_packed_f32(const float *d_grad_dist, const int32_t *d_path, const float *d_dist,
                                float *d_grad_w, const int32_t *d_n, const int64_t *d_off,
                                int32_t num_graphs, int32_t *d_status, void *stream);

/* ------------------------------------------------------------------------
 * Phase timing (a measurement hook; the paper times whole runs only, §4.1).
 * apsp_profile_enable(1) clears earlier records and starts bracketing every
 * launch of apsp_fw_f32/apsp_fw_f64 with two CUDA events on the launch
 * stream; apsp_profile_enable(0) stops recording (records are kept).
 * apsp_profile_collect waits for the recorded events and returns, per phase
 * index (0 = path init, 1 = phase 1 diagonal block, 2 = phases 2+3 panels,
 * 3 = phase 4 min-plus), the summed device time in ms and the launch count.
 * ms and launches must point to 4 entries each.  Not for use while a CUDA
 * graph is being captured.
 * ---------------------------------------------------------------------- */
int apsp_profile_enable(int on);
int apsp_profile_collect(double *ms, int64_t *launches);

/* The same records one by one, in launch order (per-round timing: the r-th
 * phase-4 record is round r of the last solve when one solve was recorded).
 * Waits for the recorded events; writes min(cap, records) entries to
 * phase[] (index as above) and ms[] (device time of that launch), and the
 * number of records to *count.  phase and ms may be NULL when cap is 0.
 * Returns APSP_EINVAL for a NULL count, a negative cap, or NULL arrays with
 * cap > 0. */
int apsp_profile_records(int32_t *phase, float *ms, int64_t cap, int64_t *count);

/* Measured ceiling of the relaxation on this GPU (a measurement hook; the
 * paper quotes datasheet peaks only, Table 1): runs the inner-loop
 * instruction pair of the FP32 kernels (dtype_bytes = 4: packed add.rn.f32x2
 * + three-input min) or of the FP64 path's lower-bound loop (dtype_bytes = 8:
 * add.rm.f32x2 + three-input min), or the integer alternative (dtype_bytes =
 * -4: one DPX fused add-then-min, __viaddmin_s32, per relaxation) on
 * registers only, on every SM, and writes the relaxations per clock per SM it
 * sustains.  Synchronises `stream`; uses and frees stream-ordered scratch.
 * Returns APSP_EINVAL for other dtype_bytes or a NULL output. */
int apsp_measure_peak(int dtype_bytes, double *relax_per_clk_per_sm, void *stream);

/* Synchronizes `stream`, then returns and clears the error words that the
 * single-graph kernels set on the device when one of their bounded waits for
 * an asynchronous copy runs out (the kernel then leaves its block unchanged,
 * so the result of that solve is incomplete): APSP_OK if no wait ran out
 * since the last call, APSP_ETIMEOUT if one did, APSP_EUNSUPPORTED if
 * apsp_fw_i32 saturated a distance, APSP_ECUDA if the stream or the
 * read-back failed. */
int apsp_device_status(void *stream);

/* Self-test of that timeout path (a test hook; the paper has no counterpart).
 * Enqueues on `stream` one small kernel that waits, with the bounded mbarrier
 * wait of the bulk-copy kernels, on a barrier that nothing completes; after
 * `polls` polls (1 .. 2^22) the wait gives up and the kernel records
 * APSP_ETIMEOUT exactly as a product kernel would, then returns.  Nothing
 * faults and the context stays usable: the next apsp_device_status returns
 * APSP_ETIMEOUT and clears it.  Returns APSP_EINVAL for polls out of range. */
int apsp_wait_timeout_selftest(uint32_t polls, void *stream);

/* Negative-cycle check of a solved matrix (§2.2 assumes no negative cycle;
 * Floyd-Warshall leaves D[i][i] < 0 on every vertex of one).  Scans the
 * diagonal of the n x n matrix d_dist (elem_bytes 4: float, 8: double; leading
 * dimension ld) after the work already on `stream`, synchronizes `stream`, and
 * returns APSP_ENEGCYCLE if some D[i][i] < 0, else APSP_OK.  With a negative
 * cycle the other distances and P are not meaningful.  Uses one fixed device
 * word of the library (calls from several host threads are serialised by a
 * lock); allocates nothing; not for use while `stream` is being captured. */
int apsp_check_negative_cycle(const void *d_dist, int elem_bytes, int64_t n, int64_t ld, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* APSP_FW_H */
