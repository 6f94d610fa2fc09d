/*
 * gna.h -- C ABI of the GB300 (sm_103a) graph-neural-ansatz variational Monte Carlo
 * library, libgna.so.
 *
 * The method is that of Yang, Hu & Li, "Scalable variational Monte Carlo with graph
 * neural ansatz", arXiv:2011.12453:
 *   - the GCN wavefunction of Eq. (gcn) with the embedding and readout described in the
 *     GNA section (two readout units: Re and Im of log Psi, the two-head form of the
 *     conclusion);
 *   - the local energy E_x = sum_x' H_xx' Psi_x'/Psi_x and MCMC sampling of
 *     P ~ |Psi|^2 of the scaling section, for the Heisenberg model
 *     H = sum_<ij> J_ij S_i . S_j and, through per-bond XXZ coefficients, the hard-core
 *     bosons of the numerical-experiments section;
 *   - the ISGO importance-reweighted gradient of Eq. (isgo).
 *
 * Conventions shared by every call:
 *   - All array arguments marked "dev" are device pointers into memory the caller
 *     allocated on the device current at the call (for example PyTorch tensors); the
 *     library never frees or retains them.  Arrays marked "host" are host pointers.
 *   - Calls that launch work are asynchronous on the given stream (0 = legacy default
 *     stream) and return once the work is enqueued.  Argument errors are detected on the
 *     host before anything is enqueued.  A kernel launch error is reported as
 *     GNA_ERR_CUDA.
 *   - The library owns only the opaque graph handle (create/destroy).  Handles are
 *     immutable after creation and may be shared by host threads and streams.  A handle
 *     lives on the device that was current when it was created; calls with it must run
 *     with that device current.
 *   - Scratch memory is supplied by the caller: each launching call takes a workspace
 *     pointer and its size in bytes, queried with gna_workspace_size().  Calls that
 *     overlap in time on the GPU must use distinct workspaces.
 *   - Spins are int8 +1 / -1, one row of n_sites per configuration.  Site numbering is
 *     that of the edge list given to gna_graph_create().
 *   - Every call returns gna_status: 0 = OK, < 0 error, > 0 warning.  No exception or
 *     abort crosses the ABI.
 */
#ifndef GNA_H
#define GNA_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define GNA_API __attribute__((visibility("default")))
#else
#define GNA_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t gna_status;
#define GNA_OK 0
#define GNA_ERR_INVALID_ARG (-1)   /* bad shape, index, null pointer, unsupported combination */
#define GNA_ERR_CUDA (-2)          /* a CUDA runtime call or kernel launch failed */
#define GNA_ERR_TIMEOUT (-3)       /* a bounded device-side wait gave up (device status word) */
#define GNA_ERR_NONFINITE (-4)     /* a non-finite value was produced (device status word) */
#define GNA_ERR_WORKSPACE (-5)     /* the workspace is smaller than gna_workspace_size() */
#define GNA_ERR_UNSUPPORTED (-6)   /* a valid request the library does not implement */
#define GNA_WARN_DEGENERATE_WEIGHTS 1 /* ISGO effective sample size below 1% of the batch
                                         (reported by gna_device_status) */

/* Arithmetic of a call.  FP64: float64 everywhere (parity path).  FP32: float32
 * features, GEMMs and ratios.  BF16: the node-feature GEMM operands in bfloat16 on the
 * tensor cores with float32 accumulation; everything else as FP32.  BF16X2: the same
 * tensor-core GEMMs with every float32 operand x carried as two bfloat16 values,
 * hi = bf16(x) and lo = bf16(x - hi) (about 16 significant bits), both multiplied and
 * accumulated in float32; feature rows in float32 and tanh to float32 accuracy.  W is a
 * bfloat16 model parameter in both tensor-core modes (the float32 theta is rounded).  The
 * backward (gna_backward) always splits its operands; the sampler runs BF16 for both.
 * Reductions across samples (energies, weights, gradients) are float64 in every mode. */
typedef enum { GNA_PREC_FP64 = 0, GNA_PREC_FP32 = 1, GNA_PREC_BF16 = 2, GNA_PREC_BF16X2 = 3 } gna_prec;

/* Nonlinearity f of Eq. (gcn), also applied after the embedding's dense layer.
 * TANH: tanh elementwise.  RELU_LN: the GNA section's f, ReLU followed by a layer
 * normalisation over the F features of each site's row, (r - mean r)/sqrt(var r + 1e-6)
 * with r = max(y, 0) and no affine part (the paper gives neither eps nor an affine part).
 * RELU_LN runs at GNA_PREC_FP64 / GNA_PREC_FP32 (calls with GNA_PREC_BF16 or BF16X2 return
 * GNA_ERR_UNSUPPORTED); its Metropolis sweeps take the one-chain-per-CTA kernel. */
typedef enum { GNA_ACT_TANH = 0, GNA_ACT_RELU_LN = 1 } gna_act;

/* Local-energy evaluation: FULL re-evaluates log Psi of every exchanged configuration
 * (one full GCN forward per antiparallel bond); INCREMENTAL recomputes only the rows of
 * the L-hop neighbourhood of the exchanged pair, layer by layer. */
typedef enum { GNA_ELOC_FULL = 0, GNA_ELOC_INCREMENTAL = 1 } gna_eloc_mode;

/* Operations whose workspace size can be queried. */
typedef enum {
  GNA_OP_FORWARD = 0,
  GNA_OP_LOCAL_ENERGY_FULL = 1,
  GNA_OP_LOCAL_ENERGY_INCREMENTAL = 2,
  GNA_OP_METROPOLIS = 3,
  GNA_OP_BACKWARD = 4,
  GNA_OP_ISGO_WEIGHTS = 5,
  GNA_OP_ISGO_GRAD = 6,
  GNA_OP_METROPOLIS_LEARNED = 7, /* gna_metropolis_sweep with a proposal network */
  GNA_OP_LOCAL_ENERGY_LOGPSI = 8 /* gna_local_energy_logpsi */
} gna_op;

/* Model description (Eq. gcn).  F = embedding width, L = number of GCN layers,
 * shared_weights = 1 for one (W, b) reused by all layers (the paper's choice),
 * 0 for one (W, b) per layer.  Limits of the library: 1 <= F <= 64 (BF16, BF16X2: F a
 * multiple of 16 and shared weights), 0 <= L <= 8, L <= the graph's max_layers. */
typedef struct {
  int32_t F;
  int32_t L;
  int32_t act;            /* gna_act */
  int32_t prec;           /* gna_prec */
  int32_t shared_weights; /* 0 or 1 */
} gna_model_desc;

typedef struct gna_graph gna_graph; /* opaque */

/* ---------------------------------------------------------------------------------
 * Library information
 * ------------------------------------------------------------------------------- */
GNA_API int32_t gna_version(void);
GNA_API const char* gna_status_string(gna_status s);

/* ---------------------------------------------------------------------------------
 * Graph.  The GNA section builds periodic boundaries into the adjacency A; here the
 * caller's edge list carries them (a bond across the boundary is an ordinary edge).
 * ------------------------------------------------------------------------------- */

/* Builds the device-resident graph: CSR adjacency, the normalised weights
 * 1/sqrt(d_i d_j) of D^-1/2 A D^-1/2 (Eq. gcn; binary A, no self-loops, couplings do
 * not enter the network), the couplings J_e, and for every bond e = (i, j) its nested
 * neighbourhoods ball_0 = {i, j}, ball_l = ball_{l-1} + neighbours, l <= max_layers,
 * used by the incremental ratio.
 *   n_sites   >= 1 (<= 4096); n_edges >= 0 (<= 1<<20)
 *   edges     host int32 [n_edges][2]: endpoints, distinct, in [0, n_sites); no
 *             duplicate bond in either orientation
 *   J         host float64 [n_edges]: coupling J_e of bond e (finite)
 *   max_layers 0..8: the largest L a model may use with this graph
 *   out       receives the handle (set to NULL on error)
 * Errors: GNA_ERR_INVALID_ARG (checked before any device call), GNA_ERR_CUDA. */
GNA_API gna_status gna_graph_create(int32_t n_sites, int32_t n_edges, const int32_t* edges,
                            const double* J, int32_t max_layers, gna_graph** out);

/* Same graph for bonds of the XXZ family.  The numerical-experiments section of the paper
 * studies hard-core bosons, H = -t sum_<ij> (b+_i b_j + h.c.) + V sum_<ij> n_i n_j; with
 * n = (1 + s)/2 and b+ <-> S+ this is, bond by bond,
 *     H_e = Jz S^z_i S^z_j + Jxy/2 (S+_i S-_j + S-_i S+_j) + hz (S^z_i + S^z_j) + c,
 * with (Jz, Jxy, hz, c) = (V, -2t, V/2, V/4).  The local energy of a configuration is then
 *     E_loc(s) = sum_e [Jz/4 s_i s_j + hz/2 (s_i + s_j) + c]
 *              + sum_{e: s_i != s_j} Jxy/2 Psi(s^e)/Psi(s).
 * Heisenberg bonds (gna_graph_create) are (J, J, 0, 0).
 *   Jz, Jxy, hz, c  host float64 [n_edges] each (finite; all four non-NULL when n_edges > 0)
 * Everything else, and the errors, as gna_graph_create.  The proposal network's coupling
 * feature is Jxy. */
GNA_API gna_status gna_graph_create_xxz(int32_t n_sites, int32_t n_edges, const int32_t* edges,
                                const double* Jz, const double* Jxy, const double* hz,
                                const double* c, int32_t max_layers, gna_graph** out);
GNA_API gna_status gna_graph_destroy(gna_graph* g);
GNA_API gna_status gna_graph_info(const gna_graph* g, int32_t* n_sites, int32_t* n_edges,
                          int32_t* max_layers);

/* Host-only: the sizes |ball_l(e)| for l = 0..n_layers of every bond, written to out
 * (host int32 [n_edges][n_layers+1]).  Same validation as gna_graph_create; makes no
 * CUDA call. */
GNA_API gna_status gna_ball_sizes_host(int32_t n_sites, int32_t n_edges, const int32_t* edges,
                               int32_t n_layers, int32_t* out);

/* ---------------------------------------------------------------------------------
 * Model
 * ------------------------------------------------------------------------------- */
GNA_API gna_status gna_model_desc_init(gna_model_desc* d, int32_t F, int32_t L, int32_t act,
                               int32_t prec, int32_t shared_weights);

/* Number of parameters P of the flat theta vector, laid out row-major as
 *   [W_e (2 x F), b_e (F), {W (2F x F), b (F)} x (shared ? 1 : L), w_r ((F+2) x 2), b_r (2)].
 * Row 0 of W_e embeds spin +1 (one-hot (1,0)), row 1 spin -1.  W rows 0..F-1 multiply
 * the message D^-1/2 A D^-1/2 H and rows F..2F-1 multiply H (the concatenation order of
 * Eq. gcn).  w_r rows 0..F-1 read the summed H^L, rows F and F+1 the summed one-hot
 * input; column 0 gives Re log Psi, column 1 Im log Psi.  Returns -1 for an invalid
 * descriptor. */
GNA_API int64_t gna_num_params(const gna_model_desc* d);

/* Workspace bytes the call `op` needs for a batch of B configurations (B = number of
 * chains for GNA_OP_METROPOLIS) on the current device.  0 is a valid answer. */
GNA_API gna_status gna_workspace_size(const gna_graph* g, const gna_model_desc* d, int32_t op,
                              int64_t B, size_t* bytes);

/* ---------------------------------------------------------------------------------
 * Compute.  theta: dev float64 [P] when d->prec == GNA_PREC_FP64, else dev float32 [P].
 * ------------------------------------------------------------------------------- */

/* log Psi(s) of a batch (Eq. gcn, embedding and readout of the GNA section).
 *   spins  dev int8 [B][n_sites]
 *   logpsi dev float64 [B][2]: (Re log Psi, Im log Psi), computed in d->prec
 * B = 0 is a no-op. */
GNA_API gna_status gna_forward(const gna_graph* g, const gna_model_desc* d, const void* theta,
                       const int8_t* spins, int64_t B, double* logpsi, void* workspace,
                       size_t workspace_bytes, void* stream);

/* Local energy of each configuration (scaling section: E_x = sum_x' H_xx' Psi_x'/Psi_x)
 * for the Heisenberg bonds of the graph:
 *   E_loc(s) = sum_e J_e/4 s_i s_j + sum_{e: s_i != s_j} J_e/2 exp(log Psi(s^e) - log Psi(s))
 * with s^e the configuration with s_i and s_j exchanged.
 *   mode   gna_eloc_mode
 *   eloc   dev float64 [B][2]: (Re, Im) of E_loc
 *   dlogpsi_bonds  dev float32 [B][n_edges] or NULL: Re(log Psi(s^e) - log Psi(s)) for
 *          antiparallel bonds, 0 for parallel ones
 * The bond ratios are formed in d->prec; the sum over bonds is float64. */
GNA_API gna_status gna_local_energy(const gna_graph* g, const gna_model_desc* d, const void* theta,
                            const int8_t* spins, int64_t B, int32_t mode, double* eloc,
                            float* dlogpsi_bonds, void* workspace, size_t workspace_bytes,
                            void* stream);

/* The incremental local energy and log Psi of each configuration in one call (the two
 * quantities an ISGO step needs at the current parameters, Eq. isgo): E_loc as
 * gna_local_energy with GNA_ELOC_INCREMENTAL, log Psi as gna_forward, both bit-identical
 * to those calls.  On the tensor cores (BF16, BF16X2) the local-energy kernel's own forward
 * gives log Psi, so the separate forward pass is not run; other precisions run both calls.
 *   eloc   dev float64 [B][2]     logpsi dev float64 [B][2]
 * Workspace: gna_workspace_size(GNA_OP_LOCAL_ENERGY_LOGPSI).  B = 0 is a no-op. */
GNA_API gna_status gna_local_energy_logpsi(const gna_graph* g, const gna_model_desc* d, const void* theta,
                                   const int8_t* spins, int64_t B, double* eloc, double* logpsi,
                                   void* workspace, size_t workspace_bytes, void* stream);

/* Metropolis(-Hastings) pair-exchange sweeps sampling P ~ |Psi|^2 (scaling section), one
 * chain per row.  Step t of chain c draws (r0, r1, r2, r3) = Philox4x64-10(key = (seed,
 * c), counter = (t, 0, 0, 0)) (Salmon et al., SC'11).
 *   Plain moves (proposal_params == NULL): bond e = hi64(r0 * n_edges); a parallel bond
 *   is a rejected step; else the exchange is accepted iff
 *   u < exp(2 Re(log Psi(s^e) - log Psi(s))), u = (r1 >> 11) 2^-53 (FP64) or
 *   (r1 >> 40) 2^-24 (FP32/BF16).
 *   Learned moves (proposal_params != NULL, network of gna_proposal_logits): with
 *   probability proposal_eps ((r3 >> 40) 2^-24 < eps) the step is a plain bond move;
 *   otherwise site i = hi64(r2 * n_sites) and its partner j is drawn from the softmax of
 *   the network's logits over i's antiparallel neighbours (uniform (r3 mod 2^32) 2^-32,
 *   neighbours in adjacency order; none: rejected step).  Either way the exchange of
 *   {i, j} is accepted iff u < exp(2 Re Delta) q(s'->s)/q(s->s') with the exact mixture
 *   density q(s->s') = (1-eps)/N [pi_i(j|s) + pi_j(i|s)] + eps/n_edges, so |Psi|^2 stays
 *   stationary.  Needs a graph of maximum degree <= 16.
 * Steps run for t = step0 .. step0 + n_sweeps*n_sites - 1.
 *   chain_spins  dev int8 [C][n_sites], read and updated in place (S_z is conserved)
 *   record_every  0 = no records; k > 0 = record after every k-th sweep
 *   proposal_params dev float32 [gna_proposal_num_params()] or NULL; proposal_eps in [0, 1]
 *   samples_out  dev int8 [n_sweeps/record_every][C][n_sites] or NULL
 *   logpsi_out   dev float64 [n_sweeps/record_every][C][2] or NULL: log Psi of each
 *                record, recomputed from the chain's state at the record
 *   n_accepted   dev int32 [C] or NULL: incremented by the number of accepted moves
 *   trace        dev float64 [C][n_sweeps*n_sites][4] or NULL: per step (bond or -1,
 *                accepted, value, kind) with value = Re Delta (plain sampler) or the log
 *                acceptance ratio (with a proposal network), NaN when nothing was
 *                proposed, and kind 1 = plain bond, 2 = network move
 * Incremental ratios are computed in d->prec; BF16 and BF16X2 models with plain moves run
 * the BF16 tensor-core sampler, with a proposal network the FP32 warp sampler. */
GNA_API gna_status gna_metropolis_sweep(const gna_graph* g, const gna_model_desc* d,
                                const void* theta, int8_t* chain_spins, int64_t C,
                                int32_t n_sweeps, int32_t record_every, uint64_t seed,
                                uint64_t step0, const float* proposal_params,
                                double proposal_eps, int8_t* samples_out, double* logpsi_out,
                                int32_t* n_accepted, double* trace, void* workspace,
                                size_t workspace_bytes, void* stream);

/* Vector-Jacobian product of log Psi (hand-written reverse mode of Eq. gcn and the
 * readout; activations are recomputed per sample, never stored across the batch):
 *   grad[k] = sum_x (cot[x][0] dRe log Psi_x/dtheta_k + cot[x][1] dIm log Psi_x/dtheta_k)
 *   cot   dev float64 [B][2]
 *   grad  dev float64 [P], overwritten
 * Per-block partial sums are reduced in float64 in a fixed order (deterministic). */
GNA_API gna_status gna_backward(const gna_graph* g, const gna_model_desc* d, const void* theta,
                        const int8_t* spins, int64_t B, const double* cot, double* grad,
                        void* workspace, size_t workspace_bytes, void* stream);

/* Same result as gna_backward, for callers that cannot allocate device memory.  The
 * paper has no counterpart: this is a deployment convenience of the library.
 *
 * Who needs it: a process whose device memory belongs to another allocator (for
 * example a framework pool that has already reserved the free memory, so a direct
 * cudaMalloc fails or fragments it), or a latency-critical loop that forbids
 * allocation after start-up because cudaMalloc may synchronise the device and take an
 * unbounded time.  This call takes no workspace and calls no cudaMalloc, cudaFree or
 * allocating library routine: its scratch (per-block gradient partials, and per-block
 * feature storage when a sample's features do not fit in shared memory) lives in a
 * fixed 32 MiB array inside the library, which every GPU that loads the library holds
 * until the process exits.
 *   Arguments and result as for gna_backward (without the workspace).
 *   The first call on a device performs a one-time set-up (it looks up the array's
 *   device address with that device current); make that first call before any stream
 *   capture.
 *   All calls share the one array, and each call overwrites what the previous one left
 *   there (nothing in it needs to start at zero).  Calls that overlap in time on the
 *   GPU -- on different streams or host threads -- race on it and give wrong results;
 *   serialise them.
 *   The block count is reduced to fit the array; a model whose single-block scratch
 *   exceeds 32 MiB is rejected with GNA_ERR_WORKSPACE. */
GNA_API gna_status gna_backward_static(const gna_graph* g, const gna_model_desc* d,
                                       const void* theta, const int8_t* spins, int64_t B,
                                       const double* cot, double* grad, void* stream);

/* ISGO weights and statistics (Eq. isgo, read as the covariance gradient):
 *   log w_x = 2 (Re logpsi_x - Re logpsi0_x) + log counts_x,  p = w / sum w (float64
 *   max-shifted log-sum-exp), Ebar = sum p E, var = sum p |E - Ebar|^2,
 *   ess = 1 / sum p^2/counts, cot_x = 2 p_x (Re(E_x - Ebar), Im(E_x - Ebar)).
 *   logpsi, logpsi0, eloc  dev float64 [B][2]
 *   counts dev float64 [B] (> 0) or NULL for all ones
 *   cot    dev float64 [B][2] or NULL
 *   stats  dev float64 [4]: (Re Ebar, Im Ebar, var, ess)
 * B >= 1.  The workspace size is given by gna_isgo_weights_workspace(). */
GNA_API gna_status gna_isgo_weights_workspace(int64_t B, size_t* bytes);
GNA_API gna_status gna_isgo_weights(const double* logpsi, const double* logpsi0, const double* eloc,
                            const double* counts, int64_t B, double* cot, double* stats,
                            void* workspace, size_t workspace_bytes, void* stream);

/* The same weights and statistics for samples sharded over several processes (the scaling
 * section's data-parallel workers: each holds a contiguous block of the chains' samples;
 * the weight sums and energies are summed across workers, then the gradient).  Two calls
 * per shard around the caller's all-reduces:
 *   gna_isgo_partials: part dev float64 [4] out = (m, S, S_re, S_im) of this shard, with
 *     m = max_x log w_x (log w as in gna_isgo_weights), S = sum_x exp(log w_x - m) and
 *     S_re + i S_im = sum_x exp(log w_x - m) E_x.
 *   The caller forms the global m (max over shards), rescales each shard's sums by
 *   exp(m_shard - m), sums them over shards to (S, S_re, S_im) and passes
 *   global = (m, S, S_re/S, S_im/S) (dev float64 [4]) to
 *   gna_isgo_finish: p = exp(log w - m)/S, cot = 2 p (E - Ebar) (dev [B][2] or NULL) and
 *     part dev float64 [3] out = (sum p |E - Ebar|^2, sum p^2/counts, sum counts) of this
 *     shard; summed over shards they give var, 1/ess and the number of copies.
 * The backward with these cotangents gives each shard's part of the gradient, summed over
 * shards by the caller.  Workspace as gna_isgo_weights_workspace(B). */
GNA_API gna_status gna_isgo_partials(const double* logpsi, const double* logpsi0, const double* eloc,
                                     const double* counts, int64_t B, double* part, void* workspace,
                                     size_t workspace_bytes, void* stream);
GNA_API gna_status gna_isgo_finish(const double* logpsi, const double* logpsi0, const double* eloc,
                                   const double* counts, int64_t B, const double* global, double* cot,
                                   double* part, void* workspace, size_t workspace_bytes, void* stream);

/* One ISGO gradient (Eq. isgo) at parameters theta on samples drawn under theta0:
 * forward log Psi, incremental local energy, weights and statistics, and the backward
 * VJP with the cotangents, all on the device.
 *   logpsi0 dev float64 [B][2]: log Psi^0 stored when the samples were drawn
 *   counts  dev float64 [B] or NULL
 *   grad    dev float64 [P]; stats dev float64 [4] as in gna_isgo_weights
 * The statistics stay on the device; nothing is synchronised. */
GNA_API gna_status isgo_grad(const gna_graph* g, const gna_model_desc* d, const void* theta,
                     const int8_t* spins, const double* logpsi0, const double* counts,
                     int64_t B, double* grad, double* stats, void* workspace,
                     size_t workspace_bytes, void* stream);

/* Grouping of duplicated samples into unique states with counts (scaling section: the
 * sampler's states are grouped before the ISGO weights, which then carry log count_x).
 *   spins     dev int8 [B][n_sites] (+-1)
 *   logpsi    dev float64 [B][2] log Psi^0 of each sample, or NULL
 *   u_spins   dev int8 [B][n_sites] out: the unique states, in order of first occurrence
 *   u_logpsi  dev float64 [B][2] out: log Psi^0 of each unique state's first occurrence
 *             (ignored when logpsi is NULL)
 *   counts    dev float64 [B] out: copies of each unique state
 *   n_unique  dev int64 [1] out: U; rows U..B-1 of the outputs are left untouched
 * Bit-exact and independent of thread scheduling.  0 <= B < 2^31, 1 <= n_sites <= 4096;
 * the workspace size is given by gna_dedup_workspace_size().  Caller-owned buffers,
 * asynchronous on stream. */
GNA_API gna_status gna_dedup_workspace_size(int64_t B, int32_t n_sites, size_t* bytes);
GNA_API gna_status gna_dedup(int32_t n_sites, const int8_t* spins, const double* logpsi, int64_t B,
                             int8_t* u_spins, double* u_logpsi, double* counts, int64_t* n_unique,
                             void* workspace, size_t workspace_bytes, void* stream);

/* Plain gradient step w <- w - lr * grad (scaling section).  theta typed as above. */
GNA_API gna_status gna_sgd_update(const gna_model_desc* d, void* theta, const double* grad,
                          double lr, void* stream);

/* ---------------------------------------------------------------------------------
 * Learned exchange proposal (not in the paper: a proposal for its MCMC step).
 * Network 9 -> 64 -> 64 -> 1 with tanh hidden units on the features of an ordered pair
 * (i, j): s_i, s_j, J_ij, 1/d_i, 1/d_j, the mean spin of i's other neighbours, that of
 * j's, and the mean over i's (j's) other neighbours u of their neighbour-spin mean.
 * Flat float32 parameters [W1 (9 x 64), b1 (64), W2 (64 x 64), b2 (64), w3 (64), b3].
 * ------------------------------------------------------------------------------- */
GNA_API int32_t gna_proposal_num_params(void);
GNA_API gna_status gna_proposal_workspace_size(const gna_graph* g, int64_t B, size_t* bytes);

/* Logits of every (configuration, bond, orientation): logits dev float32 [B][n_edges][2],
 * orientation 0 scores edges[e][0] -> edges[e][1]; NaN for parallel bonds. */
GNA_API gna_status gna_proposal_logits(const gna_graph* g, const int8_t* spins, int64_t B,
                                       const float* params, float* logits, void* stream);

/* Gradient of the training loss: mean over both orientations of every antiparallel bond
 * of (logit - min(0, 2 dlogpsi_bonds[b][e]))^2, the log acceptance of the plain move.
 *   dlogpsi_bonds dev float32 [B][n_edges] (from gna_local_energy)
 *   grad dev float64 [num_params]; loss dev float64 [1] or NULL
 * Per-block partials reduced in float64 in a fixed order. */
GNA_API gna_status gna_proposal_grad(const gna_graph* g, const int8_t* spins,
                                     const float* dlogpsi_bonds, int64_t B, const float* params,
                                     double* grad, double* loss, void* workspace,
                                     size_t workspace_bytes, void* stream);

/* One Adam step (Kingma & Ba 2015; beta1 0.9, beta2 0.999, eps 1e-8) on the float32
 * parameters with float32 moments m, v; t >= 1 is the step number. */
GNA_API gna_status gna_proposal_adam(float* params, float* m, float* v, const double* grad,
                                     int32_t t, double lr, void* stream);

/* Philox4x64-10 blocks of the sampler's generator, for bit-exact checks.
 *   keys dev uint64 [n][2]; counters dev uint64 [n][4]; out dev uint64 [n][4]. */
GNA_API gna_status gna_philox4x64_10(const uint64_t* keys, const uint64_t* counters, int64_t n,
                             uint64_t* out, void* stream);

/* Reads and optionally clears the device status word of the current device: a bit mask
 * of conditions kernels recorded since the last clear:
 *   1  a bounded device-side wait gave up (the kernel left its outputs unwritten)
 *   2  a non-finite value (ISGO statistics, or a tensor-core gradient)
 *   4  degenerate importance weights: an ISGO weighting's effective sample size
 *      1 / sum p^2/c fell below 1% of the copies in its batch (the paper warns that the
 *      gradient then explodes; resample instead of reusing the samples)
 * Kernels record these without a host synchronisation; this call synchronises the device.
 * Returns the status of the most severe condition recorded: GNA_ERR_TIMEOUT (bit 1),
 * GNA_ERR_NONFINITE (bit 2), GNA_WARN_DEGENERATE_WEIGHTS (bit 4), else GNA_OK; a failing
 * CUDA call gives GNA_ERR_CUDA and leaves *flags unset. */
GNA_API gna_status gna_device_status(int32_t* flags, int32_t clear);

/* Test hook: the iteration limit of the bounded MMA waits of the tensor-core kernels
 * launched from now on by this process (UINT32_MAX: the default, about 2 s).  With 0 every
 * such wait gives up at once: the kernel records bit 1 of the device status word, waits
 * with the default limit for the MMAs already issued, frees its tensor memory and returns,
 * so the timeout path can be tested without a fault.  Not for production use. */
GNA_API gna_status gna_debug_wait_limit(uint32_t iterations);

#ifdef __cplusplus
}
#endif
#endif /* GNA_H */
