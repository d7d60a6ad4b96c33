/*
 * dmrg.h - C ABI of the GB300 two-site ab initio DMRG hot path.
 *
 * The library computes the Davidson sigma-vector sigma = H_eff . psi of
 * two-site DMRG (Zhai & Chan, "Low communication high performance ab initio
 * DMRG algorithms": Appendix A, Eq. eff-eigsh; Sec. II.D-E for the sum over
 * normal/complementary operator pairs and its split into dense products over
 * symmetry sectors), the Davidson solve around it, and the blocking /
 * decimation / transformation steps of a sweep (Appendix A, Eqs.
 * blocked-ops and op-trans), all on one GPU with the hot path in
 * hand-written sm_103a CUDA kernels.
 *
 * Conventions shared by every entry point:
 *  - Quantum numbers are q = (N, 2Sz), compared lexicographically.
 *  - Spin orbitals are p = 2*i + sigma (alpha = 0, beta = 1); Jordan-Wigner
 *    order is ascending p; left-block modes precede right-block modes.
 *  - psi and sigma are FP64 vectors over the two-site product basis, stored
 *    block by block: blocks (q_L, q_R = Q_tot - q_L) in ascending q_L, each
 *    block row-major m_L x m_R (left index slow). dmrg_psi_layout reports
 *    the blocks.
 *  - Ownership: the caller owns every buffer it passes; the context owns all
 *    device memory it allocates (operators, work lists, scratch) until
 *    dmrg_destroy. No call keeps a caller pointer after it returns.
 *  - Pointers to psi / sigma may be host or device memory (detected with
 *    cudaPointerGetAttributes); device pointers must be on the context's
 *    device. Host buffers are copied in and out inside the call.
 *  - Streams: each context owns one CUDA stream (dmrg_stream); device work is
 *    ordered on it. Calls that return host results synchronize that stream.
 *  - Errors: every call returns a status; nothing throws across the ABI.
 *    dmrg_last_error(ctx) describes the last failure on that context.
 *  - Thread safety: one context must not be used from two threads at once;
 *    distinct contexts are independent.
 */
#ifndef DMRG_H
#define DMRG_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dmrg_ctx dmrg_ctx;

typedef enum {
  DMRG_OK = 0,
  DMRG_EINVAL = 1,   /* bad argument (size, pointer, quantum number, order of calls) */
  DMRG_ENOMEM = 2,   /* device or host allocation failed */
  DMRG_ECUDA = 3,    /* a CUDA runtime call or kernel launch failed */
  DMRG_ENOCONV = 4,  /* Davidson hit its iteration limit; best energy still returned */
  DMRG_ETIMEOUT = 5, /* a bounded device-side wait gave up */
  DMRG_ESTATE = 6    /* context not in the state the call needs (e.g. no operators loaded) */
} dmrg_status;

/* Arithmetic of the sigma products. FP64: plain double on the FP64 pipes.
 * BF16X3: every operand split into three bf16 slices x = hi + mid + lo
 * (24 significant bits); each GEMM is the sum of the 6 slice products with
 * i + j <= 2 on the tensor cores (tcgen05, FP32 accumulation, correction
 * products before the main ones); every FP32 accumulation of a sigma tile
 * spans at most dmrg_opts.tc_chain main MMA steps of 16 along K before it is
 * added into an FP32 running sum of the item. BF16X2: the
 * first two slices and the 3 products with i + j <= 1 (16 significant bits).
 * FP16X2: two fp16 slices x = hi + lo (22 significant bits) of operands
 * scaled by powers of two (each operator block and psi so that its largest
 * element lies in [2^14, 2^15)), the 3 products with i + j <= 1, FP32
 * accumulation bounded as for BF16X3; the scales are exact and undone in
 * the coefficients and the flushes. Classes whose blocks are all at most 32
 * wide run on the CUDA cores in FP32 from the same split in every mixed
 * mode. */
typedef enum { DMRG_FP64 = 0, DMRG_BF16X2 = 1, DMRG_BF16X3 = 2, DMRG_FP16X2 = 3 } dmrg_prec;

typedef struct {
  int sigma_prec;              /* dmrg_prec */
  int dav_max_space;           /* Davidson subspace size (default 24, >= 3) */
  int dav_max_iter;            /* Davidson matrix-vector products per solve (default 200) */
  int keep_one_per_q;          /* 1: in sweeps, a quantum number of psi none of whose states makes
                                  the bond-dimension cut keeps its largest one too (the kept count
                                  may exceed M; Sec. III keeps one state per quantum number) */
  double noise;                /* sweeps: decimate s psi + noise * z / |z| (renormalized), z seeded
                                  N(0,1) numbers, s = sign(psi . z); 0 = off (Sec. III runs with
                                  perturbative noise) */
  unsigned long long seed;     /* seed of the counter-based random streams (initial MPS, guesses) */
  int device;                  /* CUDA device ordinal */
  int graphs;                  /* 1: replay each sigma's launches (counter reset, product kernel,
                                  reduction; psi split for the tensor-core path) as a CUDA graph
                                  captured on the second call with the same psi / sigma pointers;
                                  0: launch them one by one. Profiling always launches directly. */
  int mixed_cut;               /* sweeps: partition of H at each bond (Sec. III.A, App. B).
                                  -1: the NC partition (Eq. h-nc) everywhere. c >= 0: mixed NC/CN -
                                  a step whose enlarged left block holds e <= c spatial orbitals uses
                                  NC, the others the CN partition (Eq. h-cn: two-index complementary
                                  operators on the left, normal ones on the right); blocks switch
                                  form by the normal-to-complementary transformation at the cut.
                                  Takes effect at dmrg_build_blocks. */
  int tc_chain;                /* tensor-core sigma: main (hi x hi) MMA steps of 16 along K that one
                                  FP32 accumulation of a sigma tile may hold before it is added into
                                  the running sum (at least one term per accumulation). The FP32
                                  rounding error of sigma grows about linearly with it. 0 = default
                                  (8 for BF16X3 and FP16X2; for BF16X2 one accumulation per
                                  64-column half of every unit of stacked terms); -1 = that
                                  unbounded setting for all three. */
  int tc_producers;            /* tensor-core sigma: warps that fill the kernel's 3-stage operand ring.
                                  1 = one warp fills every stage in order; 3 = warp w fills stage w,
                                  three stages prepared at once (faster when units hold many K
                                  stages, i.e. large blocks); 0 = default: 3 when the plan's units
                                  average 5 or more stages, else 1, until dmrg_autotune picks one.
                                  Results are bitwise the same for 1 and 3. */
} dmrg_opts;

/* Fill *o with defaults: FP64, 24, 200, 0, 0.0, seed 0, device 0, graphs 1, mixed_cut -1, tc_chain 0,
 * tc_producers 0. */
void dmrg_default_opts(dmrg_opts* o);

/* Create a context on opts->device (NULL opts = defaults). *out is NULL on failure. */
dmrg_status dmrg_create(dmrg_ctx** out, const dmrg_opts* opts);

/* Release all device memory and the stream. NULL is ignored. */
void dmrg_destroy(dmrg_ctx* ctx);

/* Message of the last failed call on ctx (static string if ctx is NULL). */
const char* dmrg_last_error(const dmrg_ctx* ctx);

/* The context's cudaStream_t, as void*. */
void* dmrg_stream(dmrg_ctx* ctx);

/* Change the sigma precision (dmrg_prec) of an existing context. Mixed modes
 * build their split operator copies (bf16 slices, 6 bytes per stored element)
 * lazily on the next dmrg_sigma call. */
dmrg_status dmrg_set_precision(dmrg_ctx* ctx, int prec);

/* Wait for all work queued on the context's stream. Returns DMRG_ETIMEOUT if
 * a tensor-core sigma launched since the last check gave up on a bounded
 * wait (its result is then invalid), DMRG_ECUDA on a CUDA error. */
dmrg_status dmrg_sync(dmrg_ctx* ctx);

/*
 * Synthetic middle-bond problem (the data-parallel hot path on its own).
 * Builds, on the device, the stored operators of an NC left block (H, a+_p,
 * R^L_p, A_pr, B_pq) and of an NC right block (H, a_p, R^R_p, P_pr, Q_pq)
 * (Appendix B, Eq. h-nc and Eq. op-def, spin-orbital U(1) form; index
 * symmetry Eq. index-sym halves the stored A/P/B/Q) over the given sector
 * lists, with every block entry N(0,1) from the counter-based SplitMix64 +
 * Box-Muller stream of `seed` (H, B_pp and Q_pp symmetric), and the NC term
 * list that pairs them.
 *   n_left_modes / n_modes: spin orbitals in the left block / in total.
 *   N, two_sz: target quantum numbers of psi.
 *   sec_left / sec_right: n*3 ints (N, 2Sz, dim) per sector, strictly
 *   ascending in (N, 2Sz), dims > 0.
 * Errors: DMRG_EINVAL for unsorted or invalid sectors, DMRG_ENOMEM when the
 * operator store does not fit in device memory.
 */
dmrg_status dmrg_load_synthetic(dmrg_ctx* ctx, int n_left_modes, int n_modes, int N, int two_sz,
                                int n_sec_left, const int* sec_left, int n_sec_right,
                                const int* sec_right, unsigned long long seed);

/*
 * One sub-Hamiltonian of the synthetic middle-bond problem, for running the
 * sigma across processes or GPUs (Sec. II.B, Eqs. sum-h, sub-h, proc-def and
 * proc-def-nc: H = sum_p H^(p), the NC terms assigned to rank p by their
 * left-block indices - one index i -> i mod n_ranks, an index pair i <= j ->
 * j(j+1)/2 + i mod n_ranks, H_L x 1 and 1 x H_R -> rank 0). Arguments as
 * dmrg_load_synthetic, plus 0 <= rank < n_ranks. The context keeps only
 * rank's terms and stores only the operators those terms use, each block
 * drawn with the same counters as in the full store (so the values equal
 * dmrg_load_synthetic's); every operator belongs to exactly one rank, so
 * each rank holds about 1/n_ranks of the operator memory. dmrg_sigma on this
 * context then returns sigma^(rank) = H_eff^(rank) psi; the sum over all
 * ranks (one all-reduce of psi_size doubles) is the full sigma.
 * dmrg_sigma_part is refused on such a context. n_ranks = 1 is
 * dmrg_load_synthetic.
 */
dmrg_status dmrg_load_synthetic_part(dmrg_ctx* ctx, int n_left_modes, int n_modes, int N, int two_sz,
                                     int n_sec_left, const int* sec_left, int n_sec_right,
                                     const int* sec_right, unsigned long long seed, int rank, int n_ranks);

/*
 * Host-only description of the partition above (no GPU or context needed):
 * for rank of n_ranks, the number of its terms, the operator elements it
 * stores, the elements of the full store (any output may be NULL), and the
 * positions of its terms in the full NC term list (the first max_ids of them
 * into term_ids; max_ids may be 0). Errors: DMRG_EINVAL for malformed
 * arguments, message via dmrg_last_error(NULL).
 */
dmrg_status dmrg_partition_info(int n_left_modes, int n_modes, int N, int two_sz, int n_sec_left,
                                const int* sec_left, int n_sec_right, const int* sec_right, int rank,
                                int n_ranks, long long* n_terms, long long* op_elements, long long* total_elements,
                                int* term_ids, int max_ids);

/*
 * Layout of psi at bond `site` (site = -1 for a synthetic context; for a
 * sweep context, the two-site step on spatial orbitals (site, site+1) with
 * the current blocks). Arrays may be NULL to query *n_blk only; otherwise
 * each must hold *n_blk entries (q_l: 2 per block). Returns the total psi
 * size in *size.
 */
dmrg_status dmrg_psi_layout(dmrg_ctx* ctx, int site, int* n_blk, int* q_l, int* m_l, int* m_r,
                            long long* offset, long long* size);

/* Work and storage figures of the current sigma: number of NC terms, of
 * (term, block) products, algorithmic FLOPs (min of the two contraction
 * orders per product, 2 per multiply-add), stored operator elements, and the
 * bytes of the operator blocks one sigma reads. */
typedef struct {
  long long n_terms;
  long long n_products;
  double flops;
  long long op_elements;
  double op_bytes_read;
  long long psi_size;
  /* tensor-core plan setting at this site for the context's precision
     (after the plan is built by a mixed-precision sigma or dmrg_autotune;
     defaults before): items per SM, producer warps, unit cost */
  int tc_items_per_sm;
  int tc_producers;
  double tc_unit_cost;
} dmrg_sigma_info;
dmrg_status dmrg_get_sigma_info(dmrg_ctx* ctx, int site, dmrg_sigma_info* info);

/*
 * sigma = H_eff . psi at bond `site` (Eq. eff-eigsh's matrix-vector product,
 * Sec. II.D-E). psi and sigma: psi_size doubles each, host or device; they
 * must not overlap. Deterministic: the same inputs give bitwise identical
 * sigma regardless of other work on the device.
 */
dmrg_status dmrg_sigma(dmrg_ctx* ctx, int site, const double* psi, double* sigma);

/*
 * Allocation-free FP64 sigma, for callers that cannot allocate device memory
 * when they need a sigma (a serving process whose HBM is fully reserved up
 * front, or a loop that must not call cudaMalloc/cudaFree because those calls
 * can block on or synchronize with other work on the device). The paper has
 * no counterpart: this is a deployment variant of dmrg_sigma.
 * Computes the same FP64 sigma as dmrg_sigma (same kernel and work list,
 * whatever the context's precision setting) but keeps the kernel's scratch
 * (partial output tiles and a work counter) in fixed-size arrays compiled
 * into the library instead of context-owned buffers; the call allocates
 * nothing. psi and sigma must be device pointers on the context's device
 * (DMRG_EINVAL for host pointers, which would need staging buffers).
 * Limits and sharing: the scratch holds at most 4,194,304 doubles (32 MiB);
 * a problem needing more is rejected with DMRG_EINVAL (use dmrg_sigma).
 * Every GPU that loads the library keeps these arrays until the process
 * exits, and all calls on a device share them: calls that overlap on the
 * GPU (other streams or contexts on the same device) race and must not be
 * issued. The first call on a device looks up the arrays' device addresses
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * The call is stream-ordered on dmrg_stream(ctx) and does not synchronize.
 */
dmrg_status dmrg_sigma_noalloc(dmrg_ctx* ctx, int site, const double* psi, double* sigma);

/*
 * Autotuner of the sigma work lists, for the context's current precision.
 * FP64: times one sigma (after one warm-up) for every combination of items
 * per SM {8, 16, 32} and per-task latency cost {4096, 16384, 65536} (the
 * item split and largest-first order of the persistent kernel's work items,
 * Sec. II.D-E collapsed into one list) on a seeded psi, keeps the fastest
 * and reports it. Mixed precision (BF16X3 / BF16X2 / FP16X2): times the
 * tensor-core path for {4, 8, 16, 32} items per SM x {1, 4, 16} x 2^20
 * multiply-adds of fixed cost per unit of stacked terms (how each output
 * tile's units are split into work items and ordered, largest first) and
 * reports the choice in items_per_sm and per_task_cost; then, unless
 * dmrg_opts.tc_producers fixes it, the other producer setting (1 or 3) on the
 * chosen plan, keeping the faster (dmrg_get_sigma_info reports it). Any output may be
 * NULL; best_ms = the chosen setting's time. Results stay bitwise deterministic for the
 * chosen setting; they can differ in the last bits from another setting
 * because items sum their terms in another grouping. A tuned FP64 work list
 * may need more scratch than dmrg_sigma_noalloc holds. Defaults without
 * tuning: FP64 8 items per SM and cost 16384; tensor cores 4 items per SM
 * and unit cost 2^20.
 */
dmrg_status dmrg_autotune(dmrg_ctx* ctx, int site, int* items_per_sm, double* per_task_cost, double* best_ms);

/*
 * One sub-Hamiltonian's share of sigma (Sec. II.B, Eqs. sum-h, sub-h,
 * proc-def, proc-def-nc, proc-def-cn): the terms of the NC sum are assigned
 * to n_ranks ranks by their left-block spin-orbital indices: one index p ->
 * p mod n_ranks; a pair p <= r -> (r(r+1)/2 + p) mod n_ranks (so O_pr and
 * O_rp, and every conjugate pair, share a rank); H_L x 1 and 1 x H_R -> rank
 * 0. At a sweep bond that uses the CN partition (dmrg_opts.mixed_cut) the
 * pair is the right-block pair of the term (Eq. proc-def-cn).
 * sigma receives the FP64 sigma of rank `rank`'s terms only; the sum over
 * ranks is the full sigma (one all-reduce of sigma in a multi-GPU setting,
 * which this library does not perform). Arguments as dmrg_sigma.
 * DMRG_EINVAL unless 0 <= rank < n_ranks.
 */
dmrg_status dmrg_sigma_part(dmrg_ctx* ctx, int site, int rank, int n_ranks, const double* psi, double* sigma);

/*
 * Lowest eigenpair of H_eff at bond `site` by Davidson (Appendix A solving
 * step; details: diagonal preconditioner clamped at 1e-8, thick restart
 * from the two lowest Ritz vectors, converged when ||H x - E x||_2^2 < tol).
 * psi0 (may be NULL = seeded random guess) and psi_out (may be NULL): host
 * or device, psi_size doubles. *iters receives the number of sigma calls.
 * DMRG_ENOCONV when dav_max_iter is reached (energy and vector still set).
 * With a mixed-precision sigma (DMRG_BF16X3 / DMRG_BF16X2) the iteration and
 * its residual use that sigma, and the returned energy is the Rayleigh
 * quotient of the final vector with one extra FP64 sigma (error second
 * order in the vector's error instead of first order in the sigma's).
 */
dmrg_status dmrg_davidson(dmrg_ctx* ctx, int site, const double* psi0, double tol, double* energy,
                          double* psi_out, int* iters);

/*
 * Full problem from integrals: t is K*K row-major (symmetric), v is K^4
 * row-major chemist's notation (ij|kl) with the 8-fold symmetry (Appendix B,
 * Eq. qc-hamil). Host pointers. Builds the initial right-canonical MPS with
 * bond dimension <= M_init (seeded) and all right-block operators
 * (blocking + transformation, right to left; NC form, or CN form right of
 * dmrg_opts.mixed_cut). Target: N electrons, 2Sz.
 */
dmrg_status dmrg_build_blocks(dmrg_ctx* ctx, const double* t, const double* v, int K, int N,
                              int two_sz, int M_init);

/*
 * Two-site sweeps (Appendix A): M_schedule[s] is the bond dimension of sweep
 * s (forward on even s, backward on odd s). energies[s] = lowest Davidson
 * energy of sweep s; max_discard[s] = largest discarded weight of sweep s
 * (either may be NULL). Davidson tolerance `tol` per step. Each solve starts
 * from the previous step's wavefunction carried to the new bond (projected
 * on the block just kept, expanded through the stored basis of the block
 * entered; at the turn of a sweep the wavefunction itself); the first step
 * after dmrg_build_blocks starts from seeded normals.
 */
dmrg_status dmrg_sweep(dmrg_ctx* ctx, const int* M_schedule, int n_sweeps, double tol,
                       double* energies, double* max_discard);

/*
 * Renormalized block operators (Eq. op-trans results) held by the context
 * after dmrg_build_blocks / dmrg_sweep, for inspection and checkpointing.
 * side 0 = left block L[j] (spin orbitals [0, 2j)), side 1 = right block
 * R[j] (spin orbitals [2j, 2K)). Operators are numbered in the canonical NC
 * order with nL = 2j: left kind H, a+_p (p < nL), R^L_p (p >= nL), A_pr
 * (p < r < nL, row-major pairs), B_pq (p <= q < nL); right kind H, a_p
 * (p >= nL), R^R_p (p < nL), P_pr, Q_pq (same pair order).
 * dmrg_block_info: *n_sectors, and when q / dims are not NULL the sectors'
 * (N, 2Sz) pairs (2 ints each) and dimensions in ascending order; *n_ops.
 * dmrg_block_read: operator `op` as a dense row-major total x total matrix
 * (total = sum of dims) over that basis, written to host memory `dense`.
 * DMRG_ESTATE when the block does not exist, DMRG_EINVAL for bad indices.
 */
dmrg_status dmrg_block_info(dmrg_ctx* ctx, int side, int j, int* n_sectors, int* q, int* dims, int* n_ops);
dmrg_status dmrg_block_read(dmrg_ctx* ctx, int side, int j, int op, double* dense);

/*
 * Per-step record of the most recent dmrg_sweep call, one entry per
 * two-site step (Appendix A steps i-iv) in execution order: sweep index,
 * bond `site` (sites site, site+1), direction (1 = forward), psi size of the
 * step, Davidson sigma calls and convergence flag, lowest energy, number of
 * states kept and discarded weight (sum of the squared singular values not
 * kept). Fills min(max_steps, available) entries of `out` (host memory,
 * may be NULL with max_steps 0) and sets *n_steps to the number available.
 */
typedef struct dmrg_step_log {
  int sweep, site, forward, iters, converged, kept;
  long long psi_size;
  double energy, discarded;
  double t_block, t_solve, t_decimate, t_transform;  /* seconds (host clock, device work included) */
} dmrg_step_log;
dmrg_status dmrg_sweep_log(dmrg_ctx* ctx, dmrg_step_log* out, int max_steps, int* n_steps);

/*
 * Serving: continuous batching of Davidson solves on one GPU (the paper
 * has no serving layer; this runs many independent Eq. eff-eigsh solves).
 * A request is a middle-bond problem with synthetic operator blocks (as
 * dmrg_load_synthetic: spin-orbital counts, target N / 2Sz, (N, 2Sz, dim)
 * sector triples, seed) plus precision, Davidson tolerance and sigma-call
 * limit. dmrg_server_submit copies the request, estimates its device
 * footprint and queues it (DMRG_ENOMEM if the footprint exceeds the
 * budget, DMRG_EINVAL for a malformed request). n_slots worker threads,
 * each with its own context and stream, admit the oldest queued request
 * whose footprint fits in the unused budget (a request passed over four
 * times blocks later ones until it fits), build its operators on the
 * device, solve, free them and post a result. dmrg_server_poll moves up to
 * max_results finished results to `out` (host), waiting up to wait_ms for
 * the first, and returns how many. Times are seconds since creation.
 * dmrg_server_destroy drops queued requests, waits for running ones and
 * frees everything. One thread at a time may call submit/poll/destroy on a
 * server.
 */
typedef struct dmrg_server dmrg_server;
typedef struct dmrg_request {
  long long id;                          /* caller's tag, copied to the result */
  int n_left_modes, n_modes, N, two_sz;  /* as dmrg_load_synthetic */
  int n_sec_left;
  const int* sec_left;
  int n_sec_right;
  const int* sec_right;
  unsigned long long seed;               /* operator blocks and Davidson guess */
  int sigma_prec;                        /* dmrg_prec */
  int max_iter;                          /* Davidson sigma-call limit */
  double tol;                            /* Davidson tolerance on ||r||^2 */
} dmrg_request;
typedef struct dmrg_result {
  long long id;
  int status;                            /* dmrg_status of the solve */
  int iters, converged, slot;
  double energy;
  double t_submit, t_admit, t_loaded, t_done;  /* t_loaded: operators built, solve starts */
  long long bytes;                       /* admitted footprint */
} dmrg_result;
dmrg_status dmrg_server_create(dmrg_server** out, int device, int n_slots, long long budget_bytes);
dmrg_status dmrg_server_submit(dmrg_server* s, const dmrg_request* r);
int dmrg_server_poll(dmrg_server* s, dmrg_result* out, int max_results, int wait_ms);
dmrg_status dmrg_server_pending(dmrg_server* s, int* queued, int* running, long long* bytes_in_use);
const char* dmrg_server_last_error(dmrg_server* s);
void dmrg_server_destroy(dmrg_server* s);

/*
 * Per-kernel timing with CUDA events recorded on the context's stream
 * around each launch of the library's kernels (tracing aid; off by default).
 * dmrg_profile(ctx, 1) clears the counters and starts recording; 2 does the
 * same and also runs the tensor-core kernel's wait accounting (which slows
 * that kernel; see dmrg_profile_waits); 0 stops.
 * dmrg_profile_read synchronizes the stream and returns, for kernel id
 * `kernel` (0 = sigma product kernels, 1 = sigma reduction, 2 = Davidson
 * vector kernels, 3 = blocking / transformation kernels, 4 = the CUDA-core
 * kernels of the mixed-precision sigma's small classes, also counted in 0),
 * the summed duration in ms and the number of launches. DMRG_EINVAL for
 * unknown ids.
 */
dmrg_status dmrg_profile(dmrg_ctx* ctx, int enable);

/* Wait accounting of the tensor-core sigma kernel, summed over its CTAs and
 * launches since dmrg_profile(ctx, 2): cycles[k] for k < 16 = clock cycles
 * spent blocked on barrier kind k, summed over the threads that wait (1 stage
 * free, by each producer warp's lanes; 2 sigma tile free, 3 X tile free, 4
 * stage loaded, 5 second-product operand written, by the MMA warp's lanes; 6
 * X tile computed, 7 second-product operand free, 8 sigma tile computed, by
 * the epilogue's; 9-13 unit-record ring; 14 and 15 are not waits: cycles the
 * MMA-issuing thread spends issuing MMAs and committing them), cycles[16] =
 * total CTA cycles. Fills min(n, 17) entries. */
dmrg_status dmrg_profile_waits(dmrg_ctx* ctx, double* cycles, int n);
dmrg_status dmrg_profile_read(dmrg_ctx* ctx, int kernel, double* total_ms, long long* launches);

#ifdef __cplusplus
}
#endif
#endif /* DMRG_H */
