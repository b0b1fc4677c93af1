/*
 * mrb — GB300-native hot path of the block-based multiresolution (MR) method
 * for the 3D Euler equations of Hoppe, Adami & Adams, "A modular massively
 * parallel computing environment for three-dimensional multiresolution
 * simulations of compressible flows" (arXiv:2012.04385).
 *
 * C ABI of libmrb.so.  Every call is extern "C", takes plain pointers and
 * sizes, returns an int status (MRB_OK = 0) and never throws.  The message of
 * the last failure is available from mrb_last_error().
 *
 * Memory.  The block pool (all heavy per-block data) is a device arena that
 * the caller allocates and owns (size from mrb_pool_bytes) and passes to
 * mrb_init_blocks; the library never frees it.  The library allocates only
 * small internal arrays (topology, work lists, reduction scratch) and frees
 * them in mrb_destroy.  Arguments documented "device" are device pointers
 * owned by the caller; "host" pointers are ordinary host memory.
 *
 * Streams.  Every call enqueues its work on cfg.stream (a cudaStream_t, NULL =
 * legacy default stream) and returns without synchronising, except
 * mrb_remesh, mrb_list_blocks/mrb_n_blocks (host topology only), mrb_sync and
 * mrb_destroy.  Kernel-side failures set a sticky device status word that
 * mrb_sync and mrb_remesh return and mrb_status reads.
 *
 * Layouts.  A block holds 16^3 internal cells (IC) and four halo cells per
 * side (Sec. 3 of the paper), 24^3 stored cells.  Per-block arrays are
 * structure-of-arrays, variable-major: [5][z][y][x] with x fastest.  The
 * conserved variables are (rho, rho u, rho v, rho w, E); primitive inputs are
 * (rho, u, v, w, p).  Blocks are identified by 64-bit modified Morton ids
 * (Sec. 3, Eq. MortonBits/AlpacaBits): 3 bits per level (x in bit 0, y in bit
 * 1, z in bit 2), finest level in the lowest group, a headbit above the top
 * group, 7 shadow levels holding the level-0 block coordinates, and the
 * instance number in bits 56..63.  Block lists are always in ascending id
 * order, which is (instance, level, Morton) order.
 */
#ifndef MRB_H
#define MRB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define MRB_OK 0
#define MRB_EINVAL 1      /* bad argument (null, out of range, unknown id)           */
#define MRB_ENOMEM 2      /* internal allocation failed                              */
#define MRB_ECAPACITY 3   /* block pool or a list buffer too small                   */
#define MRB_ECUDA 4       /* a CUDA runtime call failed                              */
#define MRB_ETIMEOUT 5    /* a bounded device wait gave up                           */
#define MRB_ENONPHYS 6    /* non-physical state (rho <= 0, p + B <= 0 or NaN)        */

/* boundary conditions, per side x-, x+, y-, y+, z-, z+ */
#define MRB_BC_ZERO_GRADIENT 0
#define MRB_BC_PERIODIC 1
#define MRB_BC_SYMMETRY 2

/* arithmetic of the bulk reconstruction/flux work */
#define MRB_FP64 0        /* everything in FP64                                      */
#define MRB_FP32_ACC64 1  /* FP32 reconstruction and flux, FP64 state, update,
                             conservation sums and time-step reduction             */

/* reconstruction */
#define MRB_RECON_WENO5 0     /* WENO5-JS everywhere                                 */
#define MRB_RECON_LEARNED 1   /* per-face MLP chooses linear 5th order or WENO5-JS   */
#define MRB_RECON_LINEAR5 2   /* linear 5th-order upwind everywhere (tests)          */
#define MRB_RECON_TENO5 3     /* TENO5 everywhere (Fu, Hu & Adams 2016): the WENO5   */
                              /* stencils kept or dropped by a sharp cutoff C_T =    */
                              /* 1e-5 on gamma_k = (1 + tau5/(beta_k + eps))^6,      */
                              /* tau5 = |beta0 - beta2|; kept ones combined with the */
                              /* linear weights renormalised                         */
#define MRB_RECON_WENOAO53 4  /* WENO-AO(5,3) everywhere (Balsara, Garain & Shu     */
                              /* 2016): the quartic over all five cells blended with */
                              /* the three parabolas, linear weights from gamma_hi = */
                              /* gamma_lo = 0.85, WENO-Z type nonlinear weights      */
                              /* gamma_k (1 + (tau/(beta_k + 1e-12))^2)              */

/* flux scheme at a face (Sec. 2.2 lists Roe, LLF and HLLC); the learned
   selector requires MRB_FLUX_ROE */
#define MRB_FLUX_ROE 0   /* per characteristic field: Roe upwinding where the two   */
                         /* face cells' and the Roe eigenvalue share a strict sign, */
                         /* else the local Lax-Friedrichs split                     */
#define MRB_FLUX_LLF 1   /* the local Lax-Friedrichs split on every field, alpha_k  */
                         /* = max |lam_k| of the two cells sharing the face         */
#define MRB_FLUX_HLLC 2  /* characteristic variables reconstructed to the face from */
                         /* both sides, mapped back to two states, HLLC (Einfeldt   */
                         /* outer speeds); an inadmissible state (rho <= 0 or       */
                         /* p + B <= 0) falls back to the two face cells' states    */

/* refinement tags, one int8 per leaf in leaf order */
#define MRB_TAG_KEEP 0
#define MRB_TAG_REFINE 1
#define MRB_TAG_COARSEN (-1)

#define MRB_MAX_INSTANCES 256
#define MRB_MAX_LEVEL 11

typedef struct mrb_config {
  int32_t n_instances;             /* independent simulations in one pool, <= 256         */
  int32_t base_blocks[3];          /* level-0 blocks per axis, each <= 128                 */
  int32_t lmax[MRB_MAX_INSTANCES]; /* finest level per instance, <= MRB_MAX_LEVEL          */
  int32_t bc[6];                   /* MRB_BC_* per side; periodic must be set on both sides*/
  int32_t precision;               /* MRB_FP64 | MRB_FP32_ACC64                            */
  int32_t recon;                   /* MRB_RECON_*                                          */
  int32_t rk_stages;               /* Runge-Kutta stages per step: 3 (TVD-RK3, also    */
                                   /* when 0) or 2 (TVD-RK2)                           */
  int32_t flux;                    /* MRB_FLUX_*                                           */
  double domain_lo[3];             /* lower corner of the domain                           */
  double dx0;                      /* level-0 cell size (block edge = 16 dx0)              */
  double gamma, B;                 /* stiffened-gas EOS, Eq. (StiffenedGas)                */
  double cfl;                      /* CFL number k of Eq. (Cfl)                            */
  double gravity[3];               /* body force in S(U) of Eq. (Euler); zero = none       */
  double eps;                      /* detail threshold at l_max (Eq. UserEpsilon applied)  */
  double mu;                       /* dynamic viscosity of the Navier-Stokes terms (Sec.   */
                                   /* 2.1; Stokes' hypothesis, no heat conduction); 0 =    */
                                   /* Euler.  Viscous face fluxes from second-order compact*/
                                   /* gradients; the time step also obeys k dx^2 /         */
                                   /* (6 max(mu/rho)).  With MRB_FP32_ACC64 it requires     */
                                   /* MRB_RECON_WENO5 and MRB_FLUX_ROE (else EINVAL)        */
  const void* mlp_weights;         /* device, learned selector weights (see mrb_mlp_*)     */
  double mlp_tau;                  /* logit threshold of the learned selector              */
  void* stream;                    /* cudaStream_t for all work                            */
  int32_t lts;                     /* 0: every leaf steps with the finest level's Delta t; */
                                   /* 1: local time stepping (Eq. LtsTimestep): level l    */
                                   /* steps with 2^(lmax - l) Delta t_lmax within a macro  */
                                   /* step (mrb_step advances one macro step); every       */
                                   /* instance must have the same lmax (else EINVAL)       */
} mrb_config;

typedef struct mrb_ctx mrb_ctx;

/* Bytes of block pool needed for `n_slots` blocks (leaves and internal nodes
 * together).  Per block: two stage buffers with halo (2 x 5 x 24^3 doubles),
 * the u^n buffer of the RK step (5 x 16^3), six face-flux buffers
 * (6 x 5 x 16^2) and the learned selector's decision bits of the current
 * step (432 words); with precision MRB_FP32_ACC64 also FP32 primitive
 * records (rho, u, v, w, p, E) of the internal cells of both stage buffers
 * (2 x 6 x 16^3 floats), which the mixed-precision stage kernel reads instead
 * of converting the FP64 state, and the FP32 increment u^(s) - u^n of the
 * current RK stage (5 x 16^3 floats); with lts also the integrated boundary-face
 * fluxes of a macro step (6 x 5 x 16^2 doubles).  Each region 256-byte
 * aligned.  Returns 0 for a bad config. */
size_t mrb_pool_bytes(const mrb_config* cfg, int64_t n_slots);

/* Create a context: checks the config, builds the level-0 topology of every
 * instance (Alg. Initialization, "initialize topology for level l0"; all
 * level-0 blocks are leaves) inside the caller's pool (device, pool_bytes
 * bytes, 256-byte aligned).  *out receives the context.  Errors: EINVAL,
 * ECAPACITY (pool smaller than the level-0 blocks), ENOMEM, ECUDA. */
int mrb_init_blocks(const mrb_config* cfg, void* pool, size_t pool_bytes, mrb_ctx** out);

/* Number of blocks (level < 0: all levels; leaves_only: leaves only). */
int mrb_n_blocks(mrb_ctx* ctx, int32_t level, int32_t leaves_only, int64_t* n);

/* Ids (host, [cap]) and geometry (host, nullable, [cap][4] = level, X, Y, Z
 * block coordinates on that level) of the selected blocks in ascending id
 * order; *n receives the count.  ECAPACITY if cap is too small. */
int mrb_list_blocks(mrb_ctx* ctx, int32_t level, int32_t leaves_only, uint64_t* keys_host, int64_t* geo_host,
                    int64_t cap, int64_t* n);

/* Impose a state on the internal cells of the listed blocks (Alg.
 * Initialization, "impose initial condition"): prim_dev [n][5][16][16][16]
 * primitive (rho, u, v, w, p), converted with E = (p + gamma B)/(gamma - 1) +
 * rho |v|^2 / 2.  keys_host: ids of existing blocks.  EINVAL on unknown id. */
int mrb_set_state(mrb_ctx* ctx, const uint64_t* keys_host, int64_t n, const double* prim_dev);

/* Impose a conserved state (device, [n][5][16^3], the layout mrb_get_state
 * returns) on the internal cells of the listed blocks: restart from a saved
 * state continues bit for bit.  EINVAL on unknown id. */
int mrb_set_cons(mrb_ctx* ctx, const uint64_t* keys_host, int64_t n, const double* cons_dev);

/* Conserved state of the listed blocks into cons_dev: [n][5][16^3] internal
 * cells (with_halo = 0) or [n][5][24^3] stored cells (with_halo = 1). */
int mrb_get_state(mrb_ctx* ctx, const uint64_t* keys_host, int64_t n, double* cons_dev, int32_t with_halo);

/* FP32 primitive records (rho, u, v, w, p, E) of the internal cells of the
 * listed blocks, [n][6][16^3] floats into records_dev (device), as the
 * mixed-precision path keeps them (fresh = 0), or converted afresh from the
 * FP64 state with the same arithmetic (fresh = 1): the two agree bit for bit
 * whenever the records are up to date.  EINVAL in an FP64 context or on an
 * unknown id.  (Inspection of the mixed-precision path's bookkeeping.) */
int mrb_get_records(mrb_ctx* ctx, const uint64_t* keys_host, int64_t n, float* records_dev, int32_t fresh);

/* Halo fill of every node (Sec. 3, Fig. MrCommunicationMesh): a halo region
 * facing a same-level node (brother or cousin) is a copy of its internal
 * cells, one facing no same-level node is predicted from the block's parent
 * by Eq. (Prediction), and cells beyond a non-periodic domain boundary take
 * the boundary condition (zero gradient, or mirror with negated normal
 * momentum).  Levels are filled coarse to fine. */
int mrb_fill_halos(mrb_ctx* ctx);

/* Right-hand side L(U) = -sum_d dF_d/dx_l + S(U) of every leaf (Eq. Euler,
 * Sec. 2.2: characteristic WENO5-JS, Roe flux with local Lax-Friedrichs
 * fallback per field), with the jump flux correction applied (Sec. 4), into
 * rhs_dev [n_leaves][5][16^3] in leaf order.  Inspection form: the time
 * stepping uses the fused mrb_rk_stage.  Halos must be filled. */
int mrb_compute_rhs(mrb_ctx* ctx, double* rhs_dev);

/* One Runge-Kutta stage (stage = 0 .. rk_stages - 1) on every leaf, fused
 * with the right-hand side, in Shu-Osher form.  TVD-RK3: u1 = un + dt L(un),
 * u2 = 3/4 un + 1/4 (u1 + dt L(u1)), u3 = 1/3 un + 2/3 (u2 + dt L(u2));
 * TVD-RK2 (the paper's standard second-order Runge-Kutta, Sec. 5): u1 = un +
 * dt L(un), u2 = 1/2 un + 1/2 (u1 + dt L(u1)).  Followed by the jump flux
 * correction of coarse cells next to finer leaves (Sec. 4, Alg. ComputeLoop).
 * dt_dev: device [n_instances] time steps (from mrb_cfl_dt).  Halos must be
 * filled. */
int mrb_rk_stage(mrb_ctx* ctx, int32_t stage, const double* dt_dev);

/* Time step of Eq. (Cfl) per instance: dt = CFL dx_lmax /
 * (max|u|+c + max|v|+c + max|w|+c) over the internal cells of its leaves,
 * into dt_dev (device, [n_instances]).  The maxima are exact. */
int mrb_cfl_dt(mrb_ctx* ctx, double* dt_dev);

/* Averaging, Eq. (Averaging): every internal node's cells become the mean of
 * their eight children, levels fine to coarse. */
int mrb_mr_project(mrb_ctx* ctx);

/* MR analysis (Eq. DetailFunction, Thresholding, LevelWiseEpsilon): for every
 * leaf at level >= 1 the details d = u - P(u_parent) over its internal and
 * halo cells (not ghost cells beyond a non-periodic boundary), block norm
 * delta = max over cells and over rho, E of |d| / |u|, threshold
 * eps_l = 2^(-3 (lmax - l)) eps.  Tags (device, [n_leaves] int8, leaf order):
 * REFINE if delta > eps_l and l < lmax (only when allow_refine), COARSEN for
 * a complete group of eight sibling leaves at level >= 2 all below eps_l
 * (with allow_refine, only if the group's parent, at level l-1, does not have
 * delta > eps_(l-1) itself: such a parent would be refined again at once, so
 * the tree would alternate from step to step), else KEEP.  delta_dev
 * (device, [n_leaves], nullable) receives delta.  Halos and the projection
 * must be current. */
int mrb_mr_predict_and_tag(mrb_ctx* ctx, int32_t allow_refine, int8_t* tags_dev, double* delta_dev);

/* Apply tags (device, [n_leaves] int8, leaf order; as from
 * mrb_mr_predict_and_tag or built by the caller): REFINE creates the eight
 * children, each predicted from the parent over its 24^3 stored cells;
 * COARSEN removes a complete sibling group (the parent already holds their
 * average).  Invalid tags (REFINE at lmax, partial COARSEN groups) are
 * ignored.  Rebuilds ids, leaf lists and the 26-neighbour table.
 * Synchronises the stream.  *n_leaves (nullable) receives the leaf count.
 * ECAPACITY when the pool has no free block left (the tree is unchanged). */
int mrb_remesh(mrb_ctx* ctx, const int8_t* tags_dev, int64_t* n_leaves);

/* Refine every leaf of `level` (Alg. Initialization: "refine all blocks of
 * level l_(m-1)" before the initial condition is imposed on level m): full
 * halo fill, then mrb_remesh with REFINE tags on those leaves.  Synchronises;
 * *n_leaves (nullable) receives the leaf count.  EINVAL for a bad level,
 * ECAPACITY as mrb_remesh. */
int mrb_refine_level(mrb_ctx* ctx, int32_t level, int64_t* n_leaves);

/* Refine the listed leaves (keys_host: ids of current leaves; restoring a
 * saved tree level by level): as mrb_refine_level.  EINVAL when an id is not
 * a leaf. */
int mrb_refine_keys(mrb_ctx* ctx, const uint64_t* keys_host, int64_t n, int64_t* n_leaves);

/* nsteps complete steps: dt from Eq. (Cfl), three fused stages each preceded
 * by the halo fill and followed by the averaging, then (when any lmax > 0)
 * halo fill, MR analysis and remesh.  dt_hist_dev (device, nullable)
 * receives [nsteps][n_instances] time steps.  The stage sequence is replayed
 * from a CUDA graph. */
int mrb_step(mrb_ctx* ctx, int32_t nsteps, double* dt_hist_dev);

/* Conserved totals per instance: sum over leaves of U dx_l^3, [n_instances][5]
 * into sums_dev (device), in a fixed reduction order. */
int mrb_sums(mrb_ctx* ctx, double* sums_dev);

/* Census of the Roe / local Lax-Friedrichs switch (Sec. 2.2, the per-field
 * rule of the MRB_FLUX_ROE scheme) for counting the algorithm's work: over
 * every face of every leaf (17 x 16 x 16 per direction), counts_host[k]
 * (host, [6]) receives the number of faces where characteristic field k
 * (0: u-c, 1: entropy, 2, 3: shear, 4: u+c) takes the LLF split rather than
 * upwinding, and counts_host[5] the number of faces.  The decisions are
 * taken in FP64 on the current stage buffer; halos must be filled.
 * Synchronous. */
int mrb_flux_census(mrb_ctx* ctx, uint64_t* counts_host);

/* Same-level neighbour ids of the listed blocks in the 26 directions
 * (index (dz+1)*9 + (dy+1)*3 + (dx+1), centre skipped), host [n][27]:
 * the id, or 0 where no same-level block exists, or 1 beyond a non-periodic
 * boundary (ids always have a headbit, so 0 and 1 are never ids). */
int mrb_neighbors(mrb_ctx* ctx, const uint64_t* keys_host, int64_t n, uint64_t* nbr_host);

/* ---- learned reconstruction selector (MRB_RECON_LEARNED) -----------------
 * Not in the paper: a 15 -> 32 -> 32 -> 1 perceptron with GELU (tanh form)
 * reads, per face, the characteristic fluxes g_m = L_k F(U_m) and variables
 * v_m = L_k U_m of fields k = 0 (u-c), 1 (entropy) and 4 (u+c) of the face's
 * Roe eigensystem over the six stencil cells m = i-2 .. i+3 -- per field the
 * five consecutive variations d = s (|g_{m+1} - g_m| + alpha_k |v_{m+1} - v_m|)
 * (alpha_k the field's local Lax-Friedrichs speed, s the sign of the flux
 * difference, of the variable difference where that is zero) compressed as
 * sign(d) log10(1 + 1e6 |d|) / 8 -- and
 * predicts whether WENO5-JS is needed (logit >= mlp_tau) or the linear
 * 5th-order upwind reconstruction suffices (logit < mlp_tau) for those three
 * fields; the shear fields always use WENO5-JS.  The selector runs at
 * stage 0 of each step (mrb_rk_stage with stage 0, and mrb_compute_rhs), on
 * the faces whose WENO5 fluxes that stage computes, and stores one decision
 * bit per face in the block pool; stages 1 and 2 apply the stored decisions
 * (a stage 1 or 2 not preceded by a stage 0 since the last remesh reads
 * decisions that belong to no state: call the stages in order).
 * Parameters: MRB_MLP_NPARAM floats (FP32 master copy, device) laid out
 * W1[32][15], b1[32], W2[32][32], b2[32], w3[32], b3; the kernels round
 * the weights to BF16 and run the layers on the tensor cores with FP32
 * accumulation.  cfg.mlp_weights points at them; the learned path applies
 * to MRB_FP32_ACC64 contexts. */
#define MRB_MLP_NPARAM 1601
#define MRB_MLP_WORK_FLOATS (512 * (MRB_MLP_NPARAM + 1))

/* Training data from the context's current state: every `stride`-th face of
 * every leaf (face id = leaf index * 13056 + direction * 4352 + position in
 * the block's face order, x then y then z faces, index f + 17 (t1 + 16 t2))
 * gives its features feats_dev [n][16] (15 + a zero pad), its label
 * labels_dev [n] (1 when, for field 0, 1 or 4 and any reconstruction the
 * face performs, |WENO5 - linear5| > max(tau_lab x the largest |input|,
 * 1e-6)) and, when
 * where_dev is not null, its face id.  n = min(cap, ceil(faces / stride)) is
 * returned in *n_out.  Halos must be filled.  FP32 arithmetic. */
int mrb_face_samples(mrb_ctx* ctx, float tau_lab, int64_t stride, float* feats_dev, uint8_t* labels_dev,
                     int64_t* where_dev, int64_t cap, int64_t* n_out);

/* Faces evaluated by the selector and faces it sent to the linear scheme
 * since the last reset (reset = 1 clears after reading).  Synchronises. */
int mrb_learned_stats(mrb_ctx* ctx, int64_t* linear_faces, int64_t* evaluated_faces, int32_t reset);

/* Selector logits of n samples (feats_dev [n][16]) on the tensor cores, into
 * logits_dev [n]; asynchronous on `stream`.  No context needed. */
int mrb_mlp_logits(const float* params_dev, const float* feats_dev, int64_t n, float* logits_dev, void* stream);

/* Threshold of the selector's decisions: the q-quantile of the logits of the
 * samples with label 1 (logits_dev [n] float, labels_dev [n] bytes, device),
 * interpolated linearly between the order statistics around position
 * (m - 1) q of the m label-1 logits in ascending order, into *tau_out (host).
 * With q = the tolerated share of label-1 faces sent to the linear scheme,
 * logit < tau selects it.  0 when no sample has label 1.  work_dev: device
 * scratch of MRB_THRESHOLD_WORK uint64.  Synchronises `stream`.  EINVAL for
 * q outside [0, 1] or null pointers with n > 0. */
#define MRB_THRESHOLD_WORK 256
int mrb_mlp_threshold(const float* logits_dev, const uint8_t* labels_dev, int64_t n, double q, uint64_t* work_dev,
                      float* tau_out, void* stream);

/* One training step of the selector on n samples: forward and backward with
 * BF16-rounded inputs, weights and hidden activations and FP32 accumulation,
 * loss = mean over samples of the binary cross-entropy with logits weighted
 * by pos_weight on label 1, gradient reduced in a fixed order, then (lr > 0)
 * one Adam step (beta 0.9, 0.999, eps 1e-8; t_step counts from 1) on the FP32
 * parameters and moments (device, MRB_MLP_NPARAM each).  work_dev: device
 * scratch of MRB_MLP_WORK_FLOATS floats.  loss_dev (device float, nullable)
 * receives the loss, grad_dev (device [MRB_MLP_NPARAM], nullable) the
 * gradient.  Asynchronous on `stream`. */
int mrb_mlp_train_step(float* params_dev, float* adam_m_dev, float* adam_v_dev, int32_t t_step, const float* feats_dev,
                       const uint8_t* labels_dev, int64_t n, float pos_weight, float lr, float* work_dev,
                       float* loss_dev, float* grad_dev, void* stream);

/* Profiling.  mrb_profile(ctx, 1) starts recording CUDA events around every
 * launch of the fused stage kernel (the dominant kernel, on cfg.stream, also
 * inside the replayed step graph) and resets the counters; 0 stops.
 * mrb_profile_read synchronises and returns the summed duration of those
 * launches (ms), their number, and the number of kernel launches the library
 * issued since profiling started (graph replays count their kernel nodes).
 * Any pointer may be null. */
int mrb_profile(mrb_ctx* ctx, int32_t enable);

/* Launch shapes (scheduling only: every choice gives bit-identical results;
 * the paper has no counterpart -- its blocks are distributed over MPI ranks).
 * params[MRB_NTUNE]: [0] stage-kernel waves (CTAs = SMs x resident CTAs per SM
 * x waves, 1..8), [1] stage work-item order (0 strided over the grid, 1 one
 * contiguous run of (block, z-slab) items per CTA), [2] region-copy halo-fill
 * CTAs per SM, [3] prediction halo-fill CTAs per SM, [4] averaging CTAs per SM
 * (1..32 each).  Defaults 1, 0, 8, 4, 8.  Per context; mrb_set_tune returns
 * EINVAL outside the ranges and re-captures the step graphs at the next
 * mrb_step. */
#define MRB_NTUNE 5
int mrb_get_tune(mrb_ctx* ctx, int32_t* params);
int mrb_set_tune(mrb_ctx* ctx, const int32_t* params);
/* Autotuner: times the candidate shapes on the context's current tree (CUDA
 * events on cfg.stream, `reps` repetitions each, after one warm-up) and keeps
 * the fastest: stage waves {1, 2, 4} x item order {0, 1}, then fill CTAs per SM
 * {4, 8, 16} x {2, 4, 8}, then averaging CTAs per SM {4, 8, 16}.  The timed work
 * leaves the simulation state unchanged: stage 0 (with the learned selector
 * also stage 1) from the current stage buffer writes only the other buffer and
 * per-step scratch, the halo fill and the averaging recompute what they wrote
 * before.  The selector's face counters (mrb_learned_stats) are reset.
 * times (host, nullable, [6]): default and tuned ms of the stage kernel(s), of
 * one halo fill and of one averaging pass.  Synchronises. */
int mrb_autotune(mrb_ctx* ctx, int32_t reps, double* times);
int mrb_profile_read(mrb_ctx* ctx, double* stage_kernel_ms, int64_t* stage_kernel_launches, int64_t* kernel_launches);

/* Conservation sums for callers that cannot allocate device memory.  (The
 * paper has no counterpart: this is a deployment variant of mrb_sums.)  Some
 * callers cannot call cudaMalloc at all -- code running under an allocator
 * that owns all device memory, or host code that must not take the driver's
 * allocation lock while other work is in flight -- so this call allocates
 * nothing: its reduction scratch is a fixed file-scope device array of
 * MRB_NOALLOC_MAX_BLOCKS x 5 doubles (2.5 MiB), held by every GPU that loads
 * the library until the process exits.
 *   blocks_dev  device, [n_blocks][5][16^3] conserved internal cells (the
 *               layout of mrb_get_state with with_halo = 0)
 *   levels_dev  device, [n_blocks] int32 level of each block (nullable: all 0)
 *   dx0         level-0 cell size; block b is weighted by (dx0 2^-level)^3
 *   stream      cudaStream_t (NULL = legacy default stream); asynchronous
 *   sums_dev    device, [5] output: sum over blocks of U dx^3, blocks in the
 *               given order, the same fixed reduction order as mrb_sums
 * With the blocks in mrb_list_blocks' leaf order the result is bitwise that
 * of mrb_sums for a single instance; n_blocks = 0 gives zeros.
 * Returns EINVAL for bad arguments, ECAPACITY for n_blocks >
 * MRB_NOALLOC_MAX_BLOCKS (nothing is launched), ECUDA on a CUDA error of this
 * call's own launches (an error pending from an earlier call is left alone).
 * Every call made outside a stream capture looks up the scratch address with
 * the calling device current (so a device reset is picked up); a call on a
 * stream being captured reuses the last address found on that device and
 * fails with ECUDA if there is none.  All calls share the scratch, which keeps
 * the last call's contents: calls that overlap on the GPU race. */
#define MRB_NOALLOC_MAX_BLOCKS 65536
int mrb_block_sums_noalloc(const double* blocks_dev, int64_t n_blocks, const int32_t* levels_dev, double dx0,
                           void* stream, double* sums_dev);

/* Throughput microbenchmarks of the current GPU (dependent-chain loops on
 * every SM): out[0] FP32 FMA TFLOP/s, out[1] FP64 FMA TFLOP/s, out[2]
 * double->float and out[3] float->double conversions (10^12 per s), out[4]
 * reciprocal square roots (10^12 per s), out[5] SM count, out[6] SM clock
 * (MHz) the device reports; with n >= 8, out[7] packed FP32 FMA
 * (fma.rn.f32x2, two FP32 FMAs per lane and instruction) TFLOP/s.  n >= 7.
 * Synchronises the device; allocates 64 bytes of scratch. */
int mrb_measure_peaks(double* out, int32_t n);

int mrb_status(mrb_ctx* ctx);   /* sticky device status (synchronises)       */
int mrb_sync(mrb_ctx* ctx);     /* synchronise the stream, return status     */
/* Reset the sticky device status to MRB_OK (after the caller has repaired or
 * replaced the offending state); synchronises.  The context stays usable. */
int mrb_clear_status(mrb_ctx* ctx);
int mrb_destroy(mrb_ctx* ctx);  /* free internal arrays (not the pool)       */
const char* mrb_last_error(mrb_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* MRB_H */
