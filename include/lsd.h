/*
 * lsd.h -- C ABI of liblsd.so: Langevin Speculative Dynamics (LSD) window
 * verification and Gaussian draft-to-target transport on one GPU.
 *
 * The method ("Speculative Sampling For Faster Molecular Dynamics"): a cheap
 * draft force field proposes a window of K second-order Langevin steps; the
 * target force field recomputes forces on every step of the window in one
 * batched evaluation; a reflection-maximal coupling of the two momentum
 * Gaussians (Eq. 5) then accepts each draft step or overrides it, and the
 * draft is rolled back to the first overridden step (Alg. 1 with lookahead
 * L = K; the per-step procedures are those of Alg. 2).  Committed states are
 * exactly distributed as plain target Langevin dynamics (Thm 3.1, Thm D.2).
 *
 * Integrator: ABOBA (Eq. 2).  The configuration text calls the scheme
 * "BAOAB"; the paper derives the coupling for ABOBA, where the force enters
 * only the mean of the BOB momentum Gaussian (Eq. 4) and the final A is a
 * shared invertible map (Thm 3.1).
 *
 * Units: Angstrom, fs, amu, eV; momentum in amu*Angstrom/fs.  A force F in
 * eV/Angstrom changes momentum at rate kappa*F with kappa = (1 eV/A)/(1
 * amu*A/fs^2) from CODATA 2018.
 *
 * Conventions for every entry point:
 *  - Return value: LSD_OK (0) or a negative LSD_E* code; lsd_strerror() names
 *    it.  No entry point aborts the process.
 *  - Ownership: the library copies every input it is given; it allocates and
 *    owns all device memory of a handle until lsd_destroy().  Output pointers
 *    are caller-owned host buffers unless the name ends in _dev, in which case
 *    they are device pointers on the handle's device.
 *  - Streams: all work of a handle is issued on one CUDA stream (the handle's
 *    own non-blocking stream unless lsd_set_stream() set another); calls that
 *    return host data synchronise that stream.
 *  - Threading: a handle is not thread-safe; distinct handles are independent.
 *  - Layouts: positions, momenta and forces are [N][3] row-major (x, y, z per
 *    atom); window arrays are [K][N][3].
 */
#ifndef LSD_H
#define LSD_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define LSD_API __attribute__((visibility("default")))
#else
#define LSD_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ------------------------------------------------------- */
#define LSD_OK 0
#define LSD_EINVAL (-1)      /* invalid argument                                  */
#define LSD_ENOMEM (-2)      /* device or host allocation failed                  */
#define LSD_ECUDA (-3)       /* a CUDA runtime call failed                        */
#define LSD_ETIMEOUT (-4)    /* a wait on the device exceeded its wall-clock limit */
#define LSD_ENONFINITE (-5)  /* a force or log-ratio was NaN or infinite          */
#define LSD_ESTATE (-6)      /* call out of order (verify without a draft, ...)   */
#define LSD_EOVERFLOW (-7)   /* a neighbour list exceeded its capacity            */
#define LSD_EUNSUPPORTED (-8) /* combination of options not built                 */

/* ---- potentials ----------------------------------------------------------
 * LSD_POT_LJ:      shifted Lennard-Jones over all periodic images within
 *                  lj_cutoff, Lorentz-Berthelot mixing of per-species eps,
 *                  sigma.
 * LSD_POT_LJ_MLP:  LJ + sum_i head(MLP(x_i)), x_i = [radial G (n_species x
 *                  n_rbf), angular G (n_ang), one-hot(species_i)], head =
 *                  head_scale*tanh(y) (LSD_HEAD_TANH) or y (LSD_HEAD_LINEAR).
 * LSD_POT_LEARNED: same form as LJ_MLP with a linear head; used as a draft
 *                  whose weights lsd_train_draft() fits by force matching.
 * Radial basis k of n_rbf: exp(-(r-mu_k)^2/(2w^2)) * (cos(pi r/rc)+1)/2 with
 * mu_k = k rc/(n_rbf-1), w = rc/(n_rbf-1), summed per neighbour species.
 * Angular term a of 16: 2^(1-zeta) (1 + lambda cos theta_ijk)^zeta
 * exp(-eta (r_ij^2 + r_ik^2)) fc(r_ij) fc(r_ik) summed over unordered
 * neighbour pairs, zeta in {1,2,4,8} (slowest index), lambda in {+1,-1},
 * eta in {0.005, 0.05} A^-2 (fastest).
 * MLP weights, packed float32: per hidden layer l: W_l [width][d_in]
 * row-major then b_l [width]; then w_out [width], b_out [1];
 * d_in = n_species*n_rbf + n_ang + n_species for the first layer.
 * Neighbour membership (the same rule everywhere, so lists are exactly
 * reproducible): positions are wrapped to 32-bit fixed point
 * u = floor(q * 2^32/L) mod 2^32 per axis.  Along an axis the pair (i, j)
 * has the wrapped difference d0 = (int32)(u_j - u_i), the minimum-image
 * displacement dmin = fl32(fl32(d0) * fl32(L/2^32)), and the image r in
 * {-1,0,1} relative to it the displacement dmin or fl32(dmin + r fl32(L));
 * the stored (absolute) image shift is s = r - k with k = (u_j - u_i -
 * d0)/2^32.  A pair is a member iff ((dx*dx + dy*dy) + dz*dz) < fl32(rc^2) in
 * binary32 without fused multiply-add; rc < L on every axis.
 */
#define LSD_POT_LJ 0
#define LSD_POT_LJ_MLP 1
#define LSD_POT_LEARNED 2

#define LSD_HEAD_TANH 0
#define LSD_HEAD_LINEAR 1

/* MLP arithmetic.  LSD_FP32 keeps FP32 accuracy on the tensor cores by
 * splitting every operand x = x_hi + x_lo and accumulating hi*hi + hi*lo +
 * lo*hi in FP32 (the dropped lo*lo term is below 2^-21 of the product).  The
 * split is in FP16 (11 significant bits each) after an exact power-of-two
 * scale: weights per layer with max|W| near 2^14, each activation and gradient
 * tensor with its |max| on the initial configuration near 2^6 (calibrated once
 * per handle, 1024x headroom to the FP16 limit).  LSD_FP32_TF32 splits in
 * TF32 instead (no scales, twice the tensor-core instructions).  Both need
 * width <= 128 and a padded input dimension <= 128; otherwise, and always for
 * LSD_FP32_CUDA_CORES, the MLP runs in plain FP32 on the CUDA cores. */
#define LSD_FP32 0            /* MLP in FP32 (tensor cores, 3 x FP16, scaled)        */
#define LSD_BF16 1            /* MLP in BF16 with FP32 accumulation                  */
#define LSD_FP8 2             /* MLP in FP8 e4m3, per-tensor scales, FP32 accumulate */
#define LSD_FP32_CUDA_CORES 3 /* MLP in FP32 on the CUDA cores                       */
#define LSD_FP32_TF32 4       /* MLP in FP32 (tensor cores, 3 x TF32)                */

typedef struct {
    int32_t n_atoms;
    int32_t n_species;
    const double *pos;          /* [N][3] Angstrom; unwrapped positions are fine          */
    const double *mom;          /* [N][3] amu*A/fs, or NULL: Maxwell-Boltzmann draw at T   */
    const int32_t *species;     /* [N], values in [0, n_species)                            */
    const double *species_mass; /* [n_species] amu, > 0                                     */
    double box[3];              /* orthorhombic periodic box, Angstrom                      */
    uint64_t seed;              /* key of the counter-based generator (Philox4x32-10)       */
} lsd_system;

typedef struct {
    int32_t kind;               /* LSD_POT_*                                                */
    int32_t precision;          /* LSD_FP32 | LSD_BF16 | LSD_FP8 | LSD_FP32_CUDA_CORES | LSD_FP32_TF32 */
    const double *lj_eps;       /* [n_species] eV                                           */
    const double *lj_sigma;     /* [n_species] Angstrom                                     */
    double lj_cutoff;           /* Angstrom; LJ term present when > 0                       */
    int32_t n_rbf, n_ang, n_layers, width;
    double desc_cutoff;         /* Angstrom                                                 */
    int32_t head;               /* LSD_HEAD_*                                               */
    double head_scale;          /* eV (0.05 for the synthetic targets)                      */
    const float *weights;       /* packed MLP parameters (see above), copied by lsd_init    */
    size_t n_weights;
} lsd_potential;

typedef struct {
    int64_t windows;            /* windows run                                              */
    int64_t committed;          /* steps committed                                          */
    int64_t rejected;           /* committed steps that were reflected (at most 1 per window)*/
    int64_t verified;           /* window steps verified (k_eff per window; staged windows:
                                   the steps up to the end of the last stage run)           */
    double sum_delta;           /* sum of |delta| (Mahalanobis, Eq. 6) over committed steps  */
    double sum_pred_reject;     /* sum of erf(|delta|/sqrt 8) over committed steps (Eq. 6)   */
    int64_t step;               /* index of the current state                               */
    int64_t stages;             /* verification passes: one per window, or per stage run     */
    int64_t list_builds;        /* Verlet-list builds asked for by the kept-list check
                                   (windows under lsd_set_list_reuse; plain target steps,
                                   which keep their lists while the evaluated positions
                                   stay within the displacement bound of their base)        */
} lsd_stats;

typedef struct lsd_handle lsd_handle;

/* lsd_init: builds a handle for the system and the two potentials, integrating
 * with ABOBA at time step dt (fs), friction gamma (1/fs) and temperature T (K),
 * window length K (1 <= K <= 128).  Derived constants (Eq. 4):
 * c1 = exp(-gamma dt); per species sigma = sqrt(m kB T kappa (1 - exp(-2 gamma
 * dt))).  Copies every input.  Errors: LSD_EINVAL (bad sizes, masses <= 0,
 * cutoff >= box, weights of the wrong length), LSD_ENOMEM, LSD_ECUDA,
 * LSD_EUNSUPPORTED. */
LSD_API int lsd_init(const lsd_system *system, const lsd_potential *draft, const lsd_potential *target, double gamma,
             double dt, double T, int32_t K, lsd_handle **out);

/* lsd_draft_window: Alg. 2 draft_step repeated K times from the current state:
 * q_mid = q + (dt/2) p/m; F~ = draft(q_mid); <p~> = c1 p + (1+c1)(dt/2) kappa F~
 * (Eq. 4); p' = <p~> + sigma xi_n with xi_n keyed by the step index n; q' =
 * q_mid + (dt/2) p'/m.  Asynchronous on the handle's stream. */
LSD_API int lsd_draft_window(lsd_handle *h);

/* lsd_verify_window: Alg. 2 verify_step on all K drafted steps at once (one
 * batched target evaluation on K*N atoms), reflectionVerify (Eq. 5) on each,
 * then the commit of Alg. 1: steps up to and including the first rejected one
 * become the new trajectory, the state is rolled to the last committed one.
 * n_committed (may be NULL) receives the number of committed steps,
 * first_reject (may be NULL) the 1-based index of the first rejected step or
 * -1.  Synchronises the stream.  LSD_ESTATE without a preceding draft. */
LSD_API int lsd_verify_window(lsd_handle *h, int32_t *n_committed, int32_t *first_reject);

/* lsd_transport_window: reflectionVerify (Eq. 5) and the commit of Alg. 1 on
 * a window given as arrays, with no draft and no target evaluation: the
 * transport step of Alg. 2 verify_step on its own.  From the current state
 * (q, p, step n0) and k <= K window steps (host buffers, [k][N][3]):
 *   q_mid    double  half-step positions A(q) of each drafted step
 *   p_draft  double  drafted momenta p'_j (p'_{j-1} is step j's input momentum)
 *   F_draft  float   draft forces F~_j at q_mid_j (eV/A; also the raw forces
 *                    of the error-correction cache)
 *   F_target float   target forces F_j at q_mid_j (eV/A)
 * z_j is the draft noise xi_{n0+j} regenerated from its counter; delta_j =
 * (1+c1)(dt/2) kappa (F~_j - F_j)/sigma; log r_j = -z.delta - |delta|^2/2 in
 * FP64; step j is accepted iff log u_{n0+j} <= min(0, log r_j).  Steps up to
 * and including the first rejected one are committed (the rejected one as
 * the reflection <p> + sigma (z - 2 (z.delta/delta.delta) delta), position
 * q_mid + (dt/2) p/m).  lsd_get_window then returns the arrays, log ratios,
 * log u and flags.  Outputs as lsd_verify_window.  Copies the inputs;
 * synchronises the stream.  LSD_EINVAL for NULL arrays or k outside
 * [1, K]. */
LSD_API int lsd_transport_window(lsd_handle *h, const double *q_mid, const double *p_draft, const float *F_draft,
                                 const float *F_target, int32_t k, int32_t *n_committed, int32_t *first_reject);

/* lsd_step: runs windows (draft + verify + commit, captured as one CUDA graph)
 * until n_steps more steps are committed; the final window commits only what
 * is needed.  stats (may be NULL) receives the cumulative counters. */
LSD_API int lsd_step(lsd_handle *h, int64_t n_steps, lsd_stats *stats);

/* lsd_plain_step: n_steps of plain target-only ABOBA Langevin from the current
 * state with the same noise keys (the baseline the metric compares against). */
LSD_API int lsd_plain_step(lsd_handle *h, int64_t n_steps);

/* lsd_set_plain_fused: plain target steps (lsd_plain_step, lsd_enqueue_plain)
 * in one cooperative launch of a fused kernel (one block per eight or four
 * atoms, the network resident in shared memory, two bounded grid barriers per
 * step) that runs every step of the call (on, the
 * default where available: ABOBA, at most 512 atoms, an
 * FP32 target network of width 32, 64 or 128 with up to 4 layers and a
 * padded input width of 32, 64 or 128, neighbour lists of capacity <= 128),
 * or as one CUDA graph of separate kernels per step (off).  The fused kernel
 * evaluates the same FP32 network on the CUDA cores (results agree with the
 * graph path to FP32 rounding).  LSD_EUNSUPPORTED when on is requested and
 * the handle's configuration has no fused plan. */
LSD_API int lsd_set_plain_fused(lsd_handle *h, int32_t on);

/* lsd_set_angular_moments: how the target's sixteen angular descriptors
 * (triplet sums over neighbour pairs, 2^(1-zeta) sum_{p<q} (1 + lambda
 * cos theta_pq)^zeta exp(-eta (r_p^2 + r_q^2)) fc_p fc_q) and their adjoint are
 * evaluated.  on: through the Cartesian moments Phi_alpha = sum_p w_p u_p^alpha
 * of the neighbour directions (the 165 monomials of degree <= 8; the pair sum
 * is (1/2)(sum_{p,q} - diagonal) of a polynomial in u_p.u_q), O(n) work per atom
 * and 1,344 bytes of moments per row (K N rows) kept from the descriptors for
 * the pair gradients.  off: the pair sums themselves, O(n^2).  Both give the
 * same functions up to FP32 rounding.  The default is on when the system's mean
 * density puts 40 or more neighbours inside the descriptor cutoff.
 * LSD_EUNSUPPORTED when the target has no angular descriptors; LSD_ENOMEM when
 * the moments cannot be allocated. */
LSD_API int lsd_set_angular_moments(lsd_handle *h, int32_t on);
/* lsd_get_angular_moments: *on = 1 when the target's angular block runs by
 * moments, else 0.  LSD_EINVAL for a null argument. */
LSD_API int lsd_get_angular_moments(const lsd_handle *h, int32_t *on);

/* lsd_set_grid_draft: the form of the draft (Alg. 2, draft_step K times) for
 * systems of at least 2048 atoms with a cell grid.  on (the default where
 * available): every draft that has the GPU to itself (lsd_draft_window, the
 * unpipelined window, the pipelined loop's first draft and redraft) runs as
 * one cooperative launch of one 512-thread CTA per SM with a bounded
 * grid-wide barrier per step (two with a learned draft); the pipelined loop's
 * speculative draft, which overlaps a verification, stays in the cluster form
 * (at most 16 SMs).  off: every draft in the cluster form.  Both forms compute
 * each atom's force in the same order and give the same bits.  A grid barrier
 * that waits more than about two seconds ends the window early and sets
 * LSD_ETIMEOUT.  LSD_EUNSUPPORTED when on is requested and the handle has no
 * grid form (fewer atoms, no cell grid, or a device that cannot co-schedule
 * the grid). */
LSD_API int lsd_set_grid_draft(lsd_handle *h, int32_t on);

/* lsd_enqueue_windows / lsd_enqueue_plain: enqueue n window graphs (or n
 * plain target steps) on the handle's stream and return without waiting;
 * windows run until the caller synchronises the stream (e.g. with CUDA events
 * around each call).  No step cap applies.  Results are read with
 * lsd_get_state / lsd_get_stats. */
LSD_API int lsd_enqueue_windows(lsd_handle *h, int32_t n_windows);
LSD_API int lsd_enqueue_plain(lsd_handle *h, int32_t n_steps);

/* lsd_get_state / lsd_set_state: host copies of the current state [N][3]
 * (pos, mom) and its step index.  Any pointer may be NULL. */
LSD_API int lsd_get_state(const lsd_handle *h, double *pos, double *mom, int64_t *step);
LSD_API int lsd_set_state(lsd_handle *h, const double *pos, const double *mom, int64_t step);

/* lsd_window_host: one window (Alg. 1, lsd_draft_window + lsd_verify_window)
 * from a host state, with the new state returned to the host, in one call:
 * the state (pos, mom [N][3], step) is copied to the device, the window runs
 * as one graph launch, and the committed state is copied back into pos_out,
 * mom_out (may alias pos, mom) with its step index and the committed count;
 * one stream synchronisation.  Pinned host buffers make the copies
 * asynchronous.  Staggered OBABO states are entered as by lsd_set_state.
 * Returns the window's error status as lsd_verify_window does. */
LSD_API int lsd_window_host(lsd_handle *h, const double *pos, const double *mom, int64_t step, double *pos_out,
                            double *mom_out, int64_t *step_out, int32_t *n_committed);

/* lsd_get_stats: cumulative counters (see lsd_stats). */
LSD_API int lsd_get_stats(const lsd_handle *h, lsd_stats *out);

/* lsd_set_stream: issue all later work on this cudaStream_t (e.g. PyTorch's
 * current stream); NULL restores the handle's own stream.  Rebuilds graphs. */
LSD_API int lsd_set_stream(lsd_handle *h, void *cuda_stream);

/* lsd_set_draft_weights: replace the draft MLP weights (packed float32, same
 * shape as at init) between windows. */
LSD_API int lsd_set_draft_weights(lsd_handle *h, const float *weights, size_t n_weights);

/* lsd_get_draft_weights: copy the current draft weights (packed float32). */
LSD_API int lsd_get_draft_weights(const lsd_handle *h, float *weights, size_t n_weights);

/* lsd_set_pipelining: 1 makes lsd_step and lsd_enqueue_windows overlap the
 * draft of window w+1 with the verification of window w (the single-GPU form
 * of the pipelined protocol of Alg. 2): while w is verified on the handle's
 * stream, a second, high-priority stream drafts w+1 speculatively from the
 * last drafted state of w into a second set of window buffers.  When w is
 * fully accepted the committed state is that speculative base bit for bit and
 * the draft is kept; otherwise w+1 is drafted again from the committed state
 * before it is verified.  Committed trajectories are identical to the
 * unpipelined loop's.  Allocates the second window buffers on first use.
 * Not with speculative error correction (the speculative draft would read the
 * cache while the commit rewrites it): returns LSD_ESTATE if EC is on, and
 * lsd_set_error_correction(h, 1) returns LSD_ESTATE while pipelining is on.
 * lsd_draft_window / lsd_verify_window / lsd_profile_window stay unpipelined. */
LSD_API int lsd_set_pipelining(lsd_handle *h, int32_t on);

/* lsd_set_window_stages: verify each window of lsd_step / lsd_enqueue_windows /
 * lsd_window_host in stages of S steps (0 < S < K; 0 or S >= K: one pass, the
 * default).  Stage s drafts steps sS .. min(K, sS + S) - 1, continuing from
 * the last drafted state, verifies them (the target forces and the transport
 * reductions of Alg. 1), and decides over every step drafted so far.  When
 * all of them are accepted, the draft reached the stage's end and the step
 * cap lies beyond it, the next stage runs: a conditional node of the window's
 * graph, set on the device, so the host does not wait.  Otherwise the window
 * commits exactly what a one-pass window commits (the first rejection and the
 * steps before it), and the steps past that stage are neither drafted nor
 * verified.  Committed trajectories and every statistic but `verified` and
 * `stages` are bit-identical to one-pass windows; per-step window arrays
 * (lsd_get_window) hold the drafted steps only.  Frames captured
 * (lsd_set_frame_capture) are the verified steps, fewer than one pass
 * verifies.  Not with pipelining: LSD_ESTATE when pipelining is on, and
 * lsd_set_pipelining(h, 1) returns LSD_ESTATE while stages are set.
 * LSD_EINVAL for S < 0. */
LSD_API int lsd_set_window_stages(lsd_handle *h, int32_t steps_per_stage);

/* lsd_set_list_reuse: 1 keeps the Verlet candidate lists of unpipelined
 * windows (lsd_step / lsd_enqueue_windows / lsd_window_host / lsd_draft_window)
 * from one window to the next: a check kernel compares the committed
 * positions with the lists' base and the lists are rebuilt only when some
 * atom has moved more than half the draft's displacement bound (0.45 skin, or
 * lsd_set_max_displacement's), or when the last draft stopped at that bound.
 * The lists stay complete for every drafted step either way (the draft checks
 * each step against the same base and ends the window at the bound), so
 * the chain is the same Markov chain; the draft's FP32 sums run over the
 * list's candidates in list order, so trajectories differ in rounding from
 * those with lists rebuilt every window.  Default 0.  Not with pipelining:
 * LSD_ESTATE when pipelining is on, and lsd_set_pipelining(h, 1) returns
 * LSD_ESTATE while reuse is on. */
LSD_API int lsd_set_list_reuse(lsd_handle *h, int32_t on);

/* lsd_set_list_skin / lsd_get_list_skin: the skin of the Verlet candidate
 * lists (list radius = the largest cutoff + skin; the draft ends a window when
 * an atom leaves 0.45 skin of the lists' base).  The handle plans it from the
 * lightest species' thermal speed over a window of K steps (1 to 2.5 A), and
 * sizes the lists' capacity and cells for that skin: a smaller skin (fewer
 * candidates per atom, lists rebuilt more often; suited to windows verified in
 * stages, which rarely draft K steps) may be set, a larger one gives
 * LSD_EINVAL.  The next windows' and plain steps' lists use it.
 * LSD_EUNSUPPORTED without cell-grid lists; lsd_get_list_skin returns 0 then. */
LSD_API int lsd_set_list_skin(lsd_handle *h, double skin);
LSD_API int lsd_get_list_skin(const lsd_handle *h, double *skin);

/* lsd_set_integrator: the Langevin splitting of the chain.
 *   LSD_ABOBA (default): Eq. 2; the state is (q, p) after a full ABOBA step.
 *   LSD_OBABO: App. E.  The chain runs in the staggered frame, whose transition
 *     is a full-step A (q += dt p/m) followed by the BOB Gaussian of Eq. 4 at
 *     the new position, verified and transported exactly as for ABOBA.  The
 *     OBABO output momentum of every committed step is recovered from the
 *     staggered momenta around it and its (already verified) target force, by
 *     drawing the first half-step noise from its conditional law (Philox
 *     stream 3 at the step index); positions are the staggered ones.  Entering
 *     the frame from an OBABO state (q, p) at step n applies the leading O and
 *     B half-steps (stream 4 at n), which costs one target force evaluation.
 * Switching to LSD_OBABO takes the current state as an OBABO state; switching
 * back takes the current OBABO output state as the ABOBA state.  Under
 * LSD_OBABO, lsd_get_state returns the OBABO output (q, p) and lsd_set_state
 * takes one (and enters the frame).  Returns LSD_EINVAL for another value. */
#define LSD_ABOBA 0
#define LSD_OBABO 1
LSD_API int lsd_set_integrator(lsd_handle *h, int32_t scheme);

/* lsd_set_max_displacement: the draft stops a window early, at the first
 * step at which some atom lies more than d_max Angstrom from the position its
 * candidate lists were built around (a stopping time: the decision depends
 * only on noise already drawn, so committed steps keep the target law).  The
 * window then verifies k_eff < K steps.  The library's own bound is 0.45
 * times the list skin (beyond it the lists could miss a pair); d_max is
 * clamped to it, and d_max = 0 restores it.  LSD_EUNSUPPORTED when the draft
 * uses no candidate lists (every atom a candidate: no displacement check). */
LSD_API int lsd_set_max_displacement(lsd_handle *h, double d_max);

/* lsd_set_error_correction: speculative error correction (Alg. 3) on (1) or
 * off (0).  On: the draft mean uses F~ + dF, where dF = F - F~raw of the last
 * committed step; switching on clears dF. */
LSD_API int lsd_set_error_correction(lsd_handle *h, int32_t on);

/* lsd_set_frame_capture: when on, every verified window step appends
 * (q_mid_j, F_target_j) to a device ring buffer of `capacity` frames used by
 * lsd_train_draft; capacity 0 turns capture off. */
LSD_API int lsd_set_frame_capture(lsd_handle *h, int64_t capacity);
LSD_API int lsd_frame_count(const lsd_handle *h, int64_t *n_frames);

/* lsd_get_frames: host copies of captured frames first .. first+count-1,
 * numbered in capture order from 0 (a window's verified steps in step order):
 * q [count][N][3] double half-step positions q_mid_j, F [count][N][3] float
 * target forces at them (either pointer may be NULL).  Only the most recent
 * `capacity` frames are held: LSD_EINVAL for a range outside them,
 * LSD_ESTATE when capture is off.  Synchronises the stream. */
LSD_API int lsd_get_frames(lsd_handle *h, int64_t first, int64_t count, double *q, float *F);

/* lsd_train_draft: n_iters Adam steps (learning rate lr) of force matching of a
 * LSD_POT_LEARNED draft on the captured frames: loss = mean over frames and
 * components of |F~ - F_target|^2, gradient by the double backward through
 * the MLP and the descriptors.  Frames of up to 256 atoms are evaluated one
 * per block; larger ones with the frame's atoms as rows of the batched
 * neighbour, descriptor and force kernels (any size; it rebuilds the
 * window's neighbour lists, so call it between windows).  loss_out (may be NULL) receives the loss of
 * the last iteration.  frames_per_iter <= 0 uses all frames. */
LSD_API int lsd_train_draft(lsd_handle *h, int32_t n_iters, float lr, int32_t frames_per_iter, float *loss_out);

/* lsd_set_online_training: retrain a LSD_POT_LEARNED draft during lsd_step
 * every `every_accepted` accepted steps (0 turns it off): between windows,
 * n_iters Adam steps (learning rate lr, frames_per_iter frames each, as
 * lsd_train_draft) on the captured target-verified frames; the next window
 * drafts with the new network (each step is still verified against the
 * target with the draft that proposed it, so the committed chain keeps the
 * target law).  lsd_step checks after each batch of windows and shortens its
 * batches to stop near the next retraining point.  Needs frame capture on
 * (LSD_ESTATE otherwise); LSD_EINVAL for a draft that is not learned. */
LSD_API int lsd_set_online_training(lsd_handle *h, int64_t every_accepted, int32_t n_iters, float lr,
                                    int32_t frames_per_iter);

/* lsd_online_status: retrainings done so far and the force-matching loss of
 * the last one ((eV/A)^2); either pointer may be NULL. */
LSD_API int lsd_online_status(const lsd_handle *h, int64_t *retrains, float *last_loss);

/* lsd_force_match_dev: loss and gradient (packed like the weights, float32) of
 * the learned draft on n_frames given frames (device pointers, positions
 * double [F][N][3], target forces float [F][N][3]); grad_dev may be NULL. */
LSD_API int lsd_force_match_dev(lsd_handle *h, const double *frames_q_dev, const float *frames_F_dev, int32_t n_frames,
                        float *loss_out, float *grad_dev);

/* lsd_target_forces_dev / lsd_draft_forces_dev: forces (float [C][N][3]) and
 * per-atom energies (float [C][N], may be NULL) of the target or draft
 * potential on C configurations (double [C][N][3], device pointers).
 * C <= K for the batched path. */
LSD_API int lsd_target_forces_dev(lsd_handle *h, const double *q_dev, int32_t n_configs, float *F_dev, float *E_atom_dev);
LSD_API int lsd_draft_forces_dev(lsd_handle *h, const double *q_dev, int32_t n_configs, float *F_dev, float *E_atom_dev);

/* lsd_neighbors: the target's neighbour lists of configuration c of the last
 * batched evaluation: keys (j << 5 | shift code, code = (sx+1)+3(sy+1)+9(sz+1))
 * in canonical order for the descriptor cutoff and the LJ cutoff.  Row stride
 * `cap`; counts [N].  Host buffers. */
LSD_API int lsd_neighbors(const lsd_handle *h, int32_t config, int32_t cap, int32_t *desc_keys, int32_t *desc_counts,
                  int32_t *lj_keys, int32_t *lj_counts);

/* lsd_descriptors: descriptors X and dE/dX ([C][N][d_in], float32, host) of
 * the last batched target evaluation (for parity checks). */
LSD_API int lsd_descriptors(const lsd_handle *h, int32_t n_configs, float *X, float *dEdX);

/* lsd_get_window: host copies of the last window's arrays, each may be NULL:
 * q_mid, p_draft [K][N][3] double; F_draft, F_target [K][N][3] float;
 * log_ratio, log_u, delta_norm [K] double; accept [K] int32. */
LSD_API int lsd_get_window(const lsd_handle *h, double *q_mid, double *p_draft, float *F_draft, float *F_target,
                   double *log_ratio, double *log_u, double *delta_norm, int32_t *accept);

/* lsd_checkpoint: serialise the full dynamical state (positions, the chain's
 * momenta -- staggered under LSD_OBABO -- and the OBABO output momenta, step,
 * seed, integrator, error-correction cache, draft weights and optimiser
 * moments) into buf; with buf == NULL only *len is set.  lsd_restore reads it
 * back into a handle built with the same system and potentials, without
 * re-entering the OBABO frame, so a restored run continues bit for bit. */
LSD_API int lsd_checkpoint(const lsd_handle *h, void *buf, size_t *len);
LSD_API int lsd_restore(lsd_handle *h, const void *buf, size_t len);

/* lsd_profile_window: runs one window (it commits like lsd_step would) with
 * its kernels issued one by one instead of as a graph, and CUDA events
 * recorded on the handle's stream between them; ms[k] receives the duration
 * of phase k for k < n_phases (at most LSD_N_PHASES):
 * 0 draft window, 1 neighbour lists, 2 descriptors, 3 MLP forward+backward,
 * 4 pair gradients + LJ, 5 force gather, 6 transport reduction,
 * 7 accept/reflect/commit, 8 the window's Verlet lists (built before the
 * draft, or checked and kept under lsd_set_list_reuse; 0 without lists).  With window stages set (lsd_set_window_stages),
 * the window profiled has the stage length S, the launch shape of a stage
 * (S drafted steps, S N verified rows).  Synchronises the stream. */
#define LSD_N_PHASES 9
LSD_API int lsd_profile_window(lsd_handle *h, double *ms, int32_t n_phases);

/* lsd_query: K, N, input dimension of the target MLP, neighbour capacities. */
LSD_API int lsd_query(const lsd_handle *h, int32_t *K, int32_t *n_atoms, int32_t *target_d_in, int32_t *nb_cap);

/* lsd_launch_counts: how many kernels of this library one window launches
 * (lsd_draft_window + lsd_verify_window, or one window of lsd_step), one round
 * of the pipelined loop (lsd_set_pipelining), and one plain step, for the
 * handle's current configuration (neighbour-list mode, transport form, MLP,
 * frame capture).  per_plain is 0 when plain steps run in the fused kernel
 * (lsd_set_plain_fused): one launch per lsd_plain_step / lsd_enqueue_plain
 * call, whatever its step count.  Memory-set nodes are not kernels and are not
 * counted.  Any pointer may be null.  No GPU work. */
LSD_API int lsd_launch_counts(const lsd_handle *h, int32_t *per_window, int32_t *per_round, int32_t *per_plain);

/* lsd_stage_launch_counts: with windows verified in stages
 * (lsd_set_window_stages), the kernels of a window's first stage (its Verlet
 * lists included) and of each later stage; a window launches
 * first + (stages run - 1) * later (lsd_stats.stages counts the stages run).
 * Without stages, first = per_window of lsd_launch_counts and later = 0.  Any
 * pointer may be null.  No GPU work. */
LSD_API int lsd_stage_launch_counts(const lsd_handle *h, int32_t *first, int32_t *later);

/* lsd_target_mlp_static_dev: the target potential's per-atom MLP (energies
 * and dE/dX) on the tensor cores, in the target's own operand arithmetic
 * (BF16, FP8 e4m3 with the handle's scales, or FP32 as three FP16 or TF32
 * products), for callers that cannot allocate device memory: code running
 * inside a host application whose own allocator owns all device memory, or a
 * latency-critical loop that must not stall on cudaMalloc's implicit device
 * synchronisation.  It allocates nothing: when the kernel needs per-CTA
 * scratch for SiLU' (layers x 128 x width x 2 bytes per CTA, when it does not
 * fit in tensor memory), that scratch is a fixed 4 MiB array inside the
 * library (held by every device that loads the library until the process
 * exits), and the kernel runs as many CTAs as the array has slots for (21 at
 * width 256 with 4 layers), each looping over its share of the 128-row tiles.
 * This entry point has no counterpart in the paper; it is the same
 * computation as the MLP step of lsd_target_forces_dev, bit for bit.
 *   X_dev     [M][d_pad] float descriptors, d_pad = target_d_in rounded up to
 *             a multiple of 32, padding columns zero (device pointer, read)
 *   E_dev     [M] float per-atom MLP energies, head included (device pointer,
 *             written)
 *   dEdX_dev  [M][d_pad] float dE/dX (device pointer, written)
 * Asynchronous on the handle's stream; the caller synchronises.  A bounded
 * wait inside the kernel that gives up sets the handle's error state, which
 * the next call that reads the handle's state reports (LSD_ETIMEOUT).  The
 * first call on a device looks up the array's device address (a one-time
 * set-up per device); make that first call before any stream capture.  Every
 * call shares the array, so calls that overlap on the GPU race; nothing in it
 * needs to start at zero.  Errors: LSD_EINVAL for NULL pointers, M < 1, or a
 * network whose SiLU' for one 128-row tile exceeds the 4 MiB array;
 * LSD_EUNSUPPORTED when the target has no MLP or its MLP runs on the CUDA
 * cores (LSD_FP32_CUDA_CORES, or FP32 wider than 128); LSD_ECUDA if the
 * launch or the address look-up fails. */
LSD_API int lsd_target_mlp_static_dev(lsd_handle *h, const float *X_dev, int32_t M, float *E_dev, float *dEdX_dev);

LSD_API void lsd_destroy(lsd_handle *h);
LSD_API const char *lsd_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* LSD_H */
