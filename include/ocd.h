/*
 * ocd.h -- C ABI of the GB300 (sm_103a) OCD soft-output MU-MIMO-OFDM detector.
 *
 * Method: optimized coordinate descent (OCD), Algorithm 1 of Wu, Dick,
 * Cavallaro, Studer, "High-Throughput Data Detection for Massive MU-MIMO-OFDM
 * using Coordinate Descent" (arXiv 1611.08779), with the max-log LLRs of Eq. 9
 * under the soft-output approximation of Section III-C.
 *
 * Problem per subcarrier w and OFDM symbol t (system model, Eq. 1):
 *     y_{w,t} = H_w s_{w,t} + n,   H_w in C^{B x U},  n ~ CN(0, N0 I_B),
 *     E|s|^2 = Es, s drawn from a Gray-labelled square QAM (or BPSK) alphabet.
 *
 * Data layout (all arrays row-major, C-contiguous, complex = interleaved
 * float32 (re, im), i.e. C99 `float _Complex` / torch.complex64):
 *     H     complex [Nsc][B][U]        channel, shared by the T symbols
 *     Y     complex [Nsc][T][B]        received vectors
 *     xhat  complex [Nsc][T][U]        equalizer output z^(K)     (optional)
 *     llr   float   [Nsc][T][U][Q]     max-log LLRs, Q = log2(order) (optional)
 * LLR bit order: for square QAM the first Q/2 bits (most significant first)
 * label the in-phase level and the next Q/2 the quadrature level, each a
 * binary-reflected Gray word over levels ordered from most negative to most
 * positive.  Sign: L > 0 favours bit 1 (Eq. 9 as printed).
 *
 * Modes (Algorithm 1, initialization): OCD_MMSE uses alpha = N0/Es and no
 * projection; OCD_BOX uses alpha = 0 and clips the real and imaginary parts
 * to [-a, a], a = sqrt(Es) * max Re{O} (Eq. 14 and Section II-D); for BPSK
 * the imaginary part is set to zero.
 *
 * Soft output (Section III-C): mu~_u = p_u = ||h_u||^2 / (||h_u||^2 + alpha),
 * rho~_u = ||h_u||^2 Es / N0 (equal to mu~/(1-mu~) in MMSE mode, and its
 * finite reading in BOX mode), LLRs taken on z_u / (mu~_u sqrt(Es)) against
 * the unit-energy alphabet.  A user whose column is zero gets z = 0, L = 0.
 *
 * Threading and ownership: device pointers are owned by the caller.  The
 * device entry points allocate nothing, never synchronize, and enqueue their
 * work on `stream` (0 = legacy default stream).  Errors are reported by the
 * return value; ocd_last_error() gives a message for the calling thread.
 * Stream order holds as for any launch: the detection kernels and the
 * unfolded form's paired kernels are launched with programmatic stream
 * serialization, so their blocks may be placed while the work ahead of them
 * in the stream drains, but they touch no global memory before it has
 * completed.
 */
#ifndef OCD_H_
#define OCD_H_

#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum { OCD_MMSE = 0, OCD_BOX = 1 } ocd_mode_t;

/*
 * Two arrangements of the same Algorithm 1 arithmetic (identical iterates in
 * exact arithmetic; both checked against the same FP64 reference):
 *   OCD_ALGO_RESIDUAL   r = y - sum_j h_j z_j kept in full (B entries per
 *                       symbol): 8B real FMAs per user update, as written.
 *   OCD_ALGO_PROJECTED  r carried as q = H^H r (U entries per symbol):
 *                       q0 = H^H y and G = H^H H once per subcarrier, then
 *                       h_u^H r = q_u and r -= h_u dz becomes q -= G[:,u] dz.
 *                       Supports U <= 8 always; U <= 16 when H and Y are
 *                       16-byte aligned with even B (float32 storage) or
 *                       B % 4 == 0 (16-bit storage); U <= 32 with float32
 *                       storage, even B and 16-byte aligned H and Y.
 *   OCD_ALGO_AUTO       PROJECTED when it supports the shape and either
 *                       T >= 2, or T == 1 with float32 storage, even B and
 *                       16-byte aligned H and Y; else RESIDUAL.
 * For T == 1 and U <= 8 (float32 storage, even B, 16-byte aligned H and Y)
 * the projected form runs with one lane per subcarrier (G and q0 accumulated
 * in registers, no reduction across lanes).  For 16 < U <= 32 and T <= 16
 * (float32 storage, even B, 16-byte aligned H and Y) its two products run on
 * the fifth-generation tensor cores with accumulators in tensor memory (one
 * CTA per SM, holding that SM's whole tensor memory while it runs); the other
 * shapes run warp-level tensor-core kernels.
 *   OCD_ALGO_PROJECTED_WARP  the projected form with warp-level tensor-core
 *                       products only.
 *   OCD_ALGO_PROJECTED_TC    the projected form with the tensor-memory kernel
 *                       for any shape it supports (16 < U <= 32, T <= 16, the
 *                       storage and alignment above); OCD_ERR_UNSUPPORTED
 *                       otherwise.
 * All projected kernels give the same results up to FP32 rounding.
 */
typedef enum {
  OCD_ALGO_AUTO = 0,
  OCD_ALGO_RESIDUAL = 1,
  OCD_ALGO_PROJECTED = 2,
  OCD_ALGO_PROJECTED_WARP = 3,
  OCD_ALGO_PROJECTED_TC = 4
} ocd_algo_t;

/*
 * Storage of H and Y (outputs are always float32): interleaved complex as
 * float32 pairs (8 bytes), or as bfloat16 / float16 pairs (4 bytes, real part
 * at the lower address).  The detector computes in float32 on the stored
 * values: products of 16-bit entries are exact in float32.
 */
typedef enum { OCD_STORE_C64 = 0, OCD_STORE_BF16 = 1, OCD_STORE_F16 = 2 } ocd_storage_t;

typedef enum {
  OCD_OK = 0,
  OCD_ERR_ARG = -1,          /* invalid argument; nothing was enqueued          */
  OCD_ERR_UNSUPPORTED = -2,  /* valid but outside the implemented limits        */
  OCD_ERR_CUDA = -3          /* a CUDA runtime call or the launch failed        */
} ocd_status_t;

/* Limits (mirroring the run-time parameters of Section IV: U <= 32, K <= 256). */
#define OCD_MAX_USERS 32
#define OCD_MAX_ANTENNAS 512
#define OCD_MAX_SWEEPS 256

/*
 * ocd_detect -- Algorithm 1 (preprocessing, K sweeps of h_u^H r, scalar
 * update with projection, residual update r -= h_u dz) followed by Eq. 9,
 * in the arrangement OCD_ALGO_AUTO picks.
 *
 *   H, Y        device pointers, layouts above.  Must not be NULL when
 *               Nsc*T > 0.  8-byte alignment is required; 16-byte alignment
 *               (and even B) enables vector loads.
 *   Nsc, T      subcarriers and symbols per subcarrier, >= 0 (0 = nothing to do).
 *   B, U        antennas 1..OCD_MAX_ANTENNAS, users 1..OCD_MAX_USERS.
 *   N0, Es      noise variance (>= 0) and symbol energy (> 0).  N0 must be
 *               > 0 when llr != NULL; N0 == 0 in MMSE mode gives plain
 *               least-squares coordinate descent.
 *   K           sweeps 0..OCD_MAX_SWEEPS (0 gives z = 0).
 *   mode        OCD_MMSE or OCD_BOX.
 *   qam_order   2 (BPSK), 4, 16, 64 or 256.
 *   xhat, llr   device outputs; either may be NULL but not both.
 * Returns OCD_OK, OCD_ERR_ARG, OCD_ERR_UNSUPPORTED or OCD_ERR_CUDA.
 */
int ocd_detect(const void* H, const void* Y, int Nsc, int B, int U, int T,
               float N0, float Es, int K, int mode, int qam_order,
               void* xhat, float* llr, cudaStream_t stream);

/*
 * ocd_detect_ex -- ocd_detect with an explicit arrangement `algo`
 * (ocd_algo_t).  ocd_detect(...) is ocd_detect_ex(..., OCD_ALGO_AUTO, stream).
 * OCD_ALGO_PROJECTED on a shape it does not support returns OCD_ERR_UNSUPPORTED.
 */
int ocd_detect_ex(const void* H, const void* Y, int Nsc, int B, int U, int T,
                  float N0, float Es, int K, int mode, int qam_order,
                  void* xhat, float* llr, int algo, cudaStream_t stream);

/*
 * ocd_detect_typed -- ocd_detect_ex for H and Y in `storage` (ocd_storage_t):
 * element size 8 bytes (OCD_STORE_C64) or 4 bytes (16-bit pairs), aligned to
 * the element size.  xhat (complex64) and llr (float32) as above.
 */
int ocd_detect_typed(const void* H, const void* Y, int storage, int Nsc, int B, int U, int T,
                     float N0, float Es, int K, int mode, int qam_order,
                     void* xhat, float* llr, int algo, cudaStream_t stream);

/*
 * ocd_detect_host -- the same computation on HOST buffers (Eq. 1 inputs in,
 * Algorithm 1 + Eq. 9 outputs out).  Copies H and Y to the caller-supplied
 * device buffers dH, dY (same sizes as H, Y), runs ocd_detect into dX / dL,
 * and copies the results back to xhat / llr on the host.  Pinned host memory
 * is needed for the copies to overlap with compute.  The subcarriers are
 * processed in `pieces` consecutive slices (1..64) so that the copies of one
 * slice overlap the kernel of another; the library uses four internal
 * streams per device, ordered after `stream` on entry and before it on exit.
 * A NULL host output skips that output (its device buffer may then be NULL).
 * Nothing is synchronized: the host results are valid once `stream` is.
 */
int ocd_detect_host(const void* H, const void* Y, int Nsc, int B, int U, int T,
                    float N0, float Es, int K, int mode, int qam_order,
                    void* xhat, float* llr,
                    void* dH, void* dY, void* dX, float* dL,
                    int pieces, cudaStream_t stream);

/*
 * ocd_fault_status -- fault word of the kernels that wait on copy engines
 * (bit 0: a wait for a bulk copy exceeded its 1 s limit; bit 1: a batched
 * launch found a cell's tensor map misaligned; in both cases the affected
 * subcarriers were left unwritten).  Returns the bits (>= 0) or
 * OCD_ERR_CUDA, and clears them when `clear` is non-zero.  Synchronizes with
 * the current device.  After a non-zero bit 0 the outputs of every launch
 * enqueued since the last check are undefined, including those of the launch
 * that follows the faulting one: a warp that gives up waits only a bounded
 * time for its own copies still in flight, and a copy that lands later may
 * overwrite shared memory the next launch's blocks are using.  Re-run those
 * launches.
 */
int ocd_fault_status(int clear);

/*
 * ocd_wait_selftest -- exercises that timeout path: enqueues one warp that
 * waits, with the same bounded wait, on a barrier nothing ever completes;
 * after limit_us microseconds (1..2000000) the wait gives up and sets bit 0
 * of the fault word.  No input or output buffer is involved.
 */
int ocd_wait_selftest(int limit_us, cudaStream_t stream);

/* ---------------------------------------------------------------------------
 * Batched form.  The paper detects one problem at a time; a base station
 * serving several cells (sectors, carriers) holds several independent
 * problems with different B, U, Nsc, T, K, mode and alphabet.  The batched
 * entry points detect a list of such problems ("cells") with persistent
 * kernels that draw their work from device ticket counters (atomicAdd only;
 * no kernel waits on another block); cells with 17-32 users and 9-16
 * symbols in the projected form run the tensor-memory kernel in a launch of
 * their own (by default: a tensor-memory launch holds whole SMs, which the
 * other cells' launches would share; PROJECTED_TC or a tune entry asks for
 * it at any T <= 16, PROJECTED_WARP not at all).
 * Each cell's results are those of ocd_detect_typed with the same arguments
 * in the same arrangement.
 * ------------------------------------------------------------------------- */

/* One cell: the arguments of ocd_detect_typed.  `algo` (ocd_algo_t):
 * OCD_ALGO_AUTO takes the tune table's choice for the cell's shape, else the
 * default (PROJECTED for float32 storage, U <= 32, even B and 16-byte
 * aligned H and Y, at any T; else RESIDUAL).  The batched PROJECTED form
 * needs exactly those conditions (OCD_ERR_UNSUPPORTED otherwise);
 * PROJECTED_WARP and PROJECTED_TC choose its kernels as for ocd_detect_ex. */
typedef struct {
  const void* H;
  const void* Y;
  void* xhat;
  float* llr;
  int storage;
  int Nsc, B, U, T;
  float N0, Es;
  int K, mode, qam_order;
  int algo;
} ocd_cell_t;

/* Tile choice for the cells of one shape (B, U, T, storage), as picked by
 * ocd_autotune_batched.  Zero fields take the defaults. */
typedef struct {
  int B, U, T, storage;  /* key */
  int algo;              /* OCD_ALGO_RESIDUAL, OCD_ALGO_PROJECTED (its default kernel),
                            OCD_ALGO_PROJECTED_WARP or OCD_ALGO_PROJECTED_TC (a cell the
                            tcgen05 kernel does not fit takes the default kernel; a cell
                            the projected form does not fit takes the residual form) */
  int symbols_per_item;  /* residual form: symbols per work item, 1 or 2 */
  int lanes_per_item;    /* residual form: lanes per work item, power of two <= 32 */
  int sc_per_ticket;     /* projected form: subcarriers per ticket, 1..256 (0 when
                            T == 1 and U <= 8: the one-lane kernel has no tile) */
  float time_us;         /* tuning measurement of this choice (informative) */
} ocd_tune_entry_t;

#define OCD_TUNE_MAX_ENTRIES 64
typedef struct {
  int n;  /* entries in use */
  ocd_tune_entry_t entry[OCD_TUNE_MAX_ENTRIES];
} ocd_tune_t;

/* Device workspace bytes a batched call over `ncells` cells needs (ticket
 * counters; a multiple of 256).  ncells < 0 gives 0. */
size_t ocd_batched_workspace_size(int ncells);

/*
 * ocd_detect_batched -- detects `ncells` cells (0..OCD_MAX_CELLS) in one
 * enqueue: a zeroing of the workspace's ticket counters, then one persistent
 * launch per kernel variant the cells need (at most 32 cells per launch;
 * a projected-form cell with T == 1 and U <= 8 gets a launch of its own of
 * the one-lane-per-subcarrier kernel), on up to four internal streams
 * ordered after `stream` on entry and before it on exit.  `workspace`: caller-owned device memory of at least
 * ocd_batched_workspace_size(ncells) bytes, 4-byte aligned, not used by
 * another call in flight.  `tune` may be NULL.  Cells with Nsc*T == 0 are
 * skipped.  Argument errors name the offending cell; nothing is enqueued
 * then.  Stream-capturable.
 */
#define OCD_MAX_CELLS 1024
int ocd_detect_batched(const ocd_cell_t* cells, int ncells, const ocd_tune_t* tune,
                       void* workspace, size_t workspace_bytes, cudaStream_t stream);

/*
 * ocd_detect_batched_static -- ocd_detect_batched for callers that cannot
 * allocate device memory: a plug-in running inside a host application that
 * owns the CUDA context and all of its memory, a process whose device memory
 * is taken up front by another allocator, or a latency-critical loop that
 * cannot afford cudaMalloc's implicit synchronization.  It takes no
 * workspace and allocates nothing (no cudaMalloc, no cudaFree, no library
 * allocation): its ticket counters live in a library-owned device array of
 * OCD_STATIC_MAX_CELLS entries (1 KiB), which every GPU that loads the
 * library holds until the process exits.  The paper has no counterpart.
 *   ncells      0..OCD_STATIC_MAX_CELLS; more gives OCD_ERR_UNSUPPORTED and
 *               nothing is enqueued.  Other arguments as ocd_detect_batched.
 * The counters are zeroed on `stream` at the start of every call.  All calls
 * on one device share them, so calls that overlap on the GPU race and give
 * wrong results: issue them on one stream, or order them with events.  The
 * first call on a device looks up the array's device address, creates the
 * library's internal streams and events for that device and sets up the
 * device's kernel attributes; make that first call before any stream capture.
 */
#define OCD_STATIC_MAX_CELLS 256
int ocd_detect_batched_static(const ocd_cell_t* cells, int ncells, const ocd_tune_t* tune,
                              cudaStream_t stream);

/*
 * ocd_autotune_batched -- builds a tune table for exactly this batch, on the
 * cells' own buffers, with `reps` timed runs (1..100) after one warm-up per
 * measurement.  Phase 1: for every distinct (B, U, T, storage), the
 * candidate tiles (each arrangement the shape supports; symbols and lanes per
 * item for the residual form, subcarriers per ticket for the projected form)
 * timed on that shape's cells alone; the fastest is kept.  Phase 2: the
 * whole batch timed at once (what the shapes' launches do to each other on
 * the internal streams), first with the defaults written out as a table,
 * then with one shape at a time changed to its other choices (the warp-level
 * or the tcgen05 kernel for 17-32 users, subcarriers per ticket halved or
 * doubled, the other arrangement); a change is kept only when the batch
 * gets more than 1.5% faster.  time_us of an entry is its shape's time
 * alone.  Writes the result to `tune` (replacing its contents).  Overwrites
 * the cells' outputs; synchronizes `stream`.  At most OCD_TUNE_MAX_ENTRIES
 * shapes.
 */
int ocd_autotune_batched(const ocd_cell_t* cells, int ncells, void* workspace,
                         size_t workspace_bytes, int reps, ocd_tune_t* tune,
                         cudaStream_t stream);

/*
 * CUDA-graph form of ocd_detect_batched: ocd_graph_create_batched captures
 * one ocd_detect_batched call (cells, tune and workspace bound at creation)
 * into an executable graph on the current device; ocd_graph_launch replays
 * it on `stream`; ocd_graph_destroy releases it (NULL is ignored).
 */
typedef struct ocd_graph ocd_graph_t;
int ocd_graph_create_batched(const ocd_cell_t* cells, int ncells, const ocd_tune_t* tune,
                             void* workspace, size_t workspace_bytes, ocd_graph_t** graph);
int ocd_graph_launch(ocd_graph_t* graph, cudaStream_t stream);
int ocd_graph_destroy(ocd_graph_t* graph);

/* ---------------------------------------------------------------------------
 * Unfolded (differentiable) form.  Not in the paper: Algorithm 1 with K fixed
 * sweeps whose regularizer alpha_k and damping omega_k are learnable per
 * sweep.  Sweep k uses d_{u,k} = 1/(||h_u||^2 + alpha_k), p_{u,k} =
 * d_{u,k} ||h_u||^2 (both 0 when the denominator is <= 0) and the update
 *     c = proj(d_{u,k} h_u^H r + p_{u,k} z_u),  dz = omega_k (c - z_u),
 *     z_u <- z_u + dz,  r <- r - h_u dz
 * (omega_k = 1 and alpha_k = alpha give Algorithm 1).  Soft output: Eq. 9
 * with mu~ = p_{u,K} and rho~ = ||h_u||^2 Es / N0[w].  The adjoint treats
 * the projection's derivative as 1 strictly inside the box and 0 on or
 * outside its bound, and passes the derivative of Eq. 9's minima to the
 * minimizing level.  H and Y are complex64 only.
 * ------------------------------------------------------------------------- */

/*
 * Arrangements (`algo`, ocd_algo_t), identical in exact arithmetic:
 *   OCD_ALGO_RESIDUAL   the residual r is carried (B entries per sample);
 *                       checkpoints: r and z at the start of every sweep,
 *                       complex64 [K][Nsc*T][B+U].
 *   OCD_ALGO_PROJECTED  q = H^H r is carried (U entries) with G = H^H H per
 *                       sample; checkpoints: G [Nsc*T][U][U], then q and z at
 *                       the start of every sweep [K][Nsc*T][2U].  Needs the
 *                       per-warp shared-memory copy of H to fit (every shape
 *                       but the largest B with large U); OCD_ERR_UNSUPPORTED
 *                       otherwise.
 *   OCD_ALGO_AUTO       PROJECTED when it fits, else RESIDUAL.
 * The forward and backward calls of one step must pass the same algo.
 */

/* Device bytes of the checkpoints of `algo` (layouts above). */
size_t ocd_unfolded_checkpoint_size(int Nsc, int B, int U, int T, int K, int algo);
/* Device workspace bytes of ocd_unfolded_backward (per-sample partial
 * gradients; a multiple of 256). */
size_t ocd_unfolded_workspace_size(int Nsc, int T, int K);

/*
 * ocd_unfolded_forward -- the unfolded sweeps and soft output.
 *   H, Y        device complex64, layouts as ocd_detect.
 *   N0          device float [Nsc]: noise variance per subcarrier (> 0 where
 *               LLRs are requested; not checked on the host).
 *   K           1..OCD_MAX_SWEEPS; omega, alpha: device float [K].
 *   xhat        device complex64 [Nsc][T][U] (required: the adjoint reads it).
 *   llr         device float [Nsc][T][U][Q] or NULL.
 *   ckpt        device buffer of ocd_unfolded_checkpoint_size(..., algo)
 *               bytes, written here and read by ocd_unfolded_backward.
 */
int ocd_unfolded_forward(const void* H, const void* Y, int Nsc, int B, int U, int T,
                         const float* N0, float Es, int K, int mode, int qam_order,
                         const float* omega, const float* alpha, void* xhat, float* llr,
                         void* ckpt, int algo, cudaStream_t stream);

/*
 * ocd_unfolded_backward -- gradients of a loss with respect to omega and
 * alpha, given its gradients with respect to xhat (dxhat, complex64
 * [Nsc][T][U], adjoint convention dl/dRe + i dl/dIm) and to the LLRs (dllr,
 * float [Nsc][T][U][Q]); either may be NULL.  H, N0, omega, alpha, xhat and
 * ckpt are those of the forward call (unchanged since; same algo).  Writes domega and
 * dalpha (device float [K]; summed over all samples in a fixed order, so the
 * result is deterministic).  workspace: ocd_unfolded_workspace_size(Nsc, T,
 * K) device bytes, 4-byte aligned.
 */
int ocd_unfolded_backward(const void* H, int Nsc, int B, int U, int T, const float* N0,
                          float Es, int K, int mode, int qam_order, const float* omega,
                          const float* alpha, const void* xhat, const void* ckpt,
                          const void* dxhat, const float* dllr, float* domega, float* dalpha,
                          void* workspace, size_t workspace_bytes, int algo, cudaStream_t stream);

/*
 * Fused training loss of the unfolded form: the mean binary cross-entropy of
 * bit labels under P(b = 1) = sigmoid(L) over all N = Nsc*T*U*Q LLRs L of
 * Eq. 9 (L > 0 favours bit 1):
 *     loss = (1/N) sum [max(L, 0) - y L + log(1 + exp(-|L|))],
 *     d loss / d L = (sigmoid(L) - y) / N,
 * computed by the forward kernel where each LLR is formed, so that no
 * separate loss kernels run between the forward and the adjoint.  The same
 * function of the LLRs as binary_cross_entropy_with_logits with mean
 * reduction.
 *
 * ocd_unfolded_bce_forward -- ocd_unfolded_forward plus the loss.
 *   bits        device float [Nsc][T][U][Q]: labels y in [0, 1], the bit
 *               order of the LLRs.
 *   llr         device float [Nsc][T][U][Q] or NULL (the LLRs themselves).
 *   dllr        device float [Nsc][T][U][Q]: d loss / d L (the adjoint input
 *               of ocd_unfolded_bce_backward).
 *   loss        device float [1]: the mean loss; 0 for an empty batch.
 *   workspace   ocd_unfolded_workspace_size(Nsc, T, K) device bytes, 4-byte
 *               aligned (per-sample loss sums, added in a fixed order: the
 *               loss is deterministic).
 * Other arguments as ocd_unfolded_forward.
 */
int ocd_unfolded_bce_forward(const void* H, const void* Y, int Nsc, int B, int U, int T,
                             const float* N0, float Es, int K, int mode, int qam_order,
                             const float* omega, const float* alpha, const float* bits,
                             void* xhat, float* llr, float* dllr, float* loss, void* ckpt,
                             void* workspace, size_t workspace_bytes, int algo,
                             cudaStream_t stream);

/*
 * ocd_unfolded_bce_backward -- d loss / d omega and d loss / d alpha of the
 * fused loss, times dloss (device float [1], the adjoint of the loss; NULL
 * means 1): ocd_unfolded_backward with dxhat = NULL and dllr the forward's
 * output, the scale applied to the summed gradients.  Arguments as
 * ocd_unfolded_backward.
 */
int ocd_unfolded_bce_backward(const void* H, int Nsc, int B, int U, int T, const float* N0,
                              float Es, int K, int mode, int qam_order, const float* omega,
                              const float* alpha, const void* xhat, const void* ckpt,
                              const float* dllr, const float* dloss, float* domega,
                              float* dalpha, void* workspace, size_t workspace_bytes, int algo,
                              cudaStream_t stream);

/* Message describing the last non-OK status returned on the calling thread. */
const char* ocd_last_error(void);

/* Library version as MAJOR*10000 + MINOR*100 + PATCH. */
int ocd_version(void);

#ifdef __cplusplus
}
#endif

#endif /* OCD_H_ */
