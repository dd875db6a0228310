// lsd_kernels.h -- host-side launchers of the kernels of liblsd.so (internal).
#pragma once
#include <cstdlib>

#include <cuda_runtime.h>

#include <utility>

#include "lsd_common.cuh"

namespace lsd {

// Launches kern as a programmatic dependent of the stream's previous kernel
// (its launch overlaps that kernel's tail).  Only for kernels that call
// pdl_wait() before touching memory an earlier kernel writes.
// Whether launch_dependent (and the cooperative transport) use programmatic
// dependent launches: the launch of the moment (a handle sets it while it
// captures its graphs), unless the environment fixes it (LSD_PDL=0 or 1, read
// once per process, for comparisons).
inline int &pdl_current() {
    static int on = 1;
    return on;
}
inline int pdl_env() {
    static const int v = [] {
        const char *e = std::getenv("LSD_PDL");
        return (e && (e[0] == '0' || e[0] == '1')) ? e[0] - '0' : -1;
    }();
    return v;
}
inline bool pdl_enabled() { return pdl_env() >= 0 ? pdl_env() != 0 : pdl_current() != 0; }

template <typename... KArgs, typename... Args>
inline void launch_dependent(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                             Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl_enabled() ? 1 : 0;
    cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

// verification (lsd_verify.cu)
void launch_fixpoint(const double *q, const int *species, int M, const Geo &g, uint4 *fix, cudaStream_t s);
void launch_neigh_build(const uint4 *fix, int M, const Geo &g, float rmax2f, float near2f, int cap_near, int cap_far,
                        int *near_keys, int *far_keys, int *n_near, int *n_far, DevState *st, cudaStream_t s,
                        const int *keff = nullptr, int j_off = 0);
// mom (may be null): [M][kMomFloats] moments of the rows; non-null selects the
// moment form of the angular features and their adjoint (the same rows of
// moments for both calls)
constexpr int kMomRowFloats = 336;
void launch_desc(const uint4 *fix, const int *near_keys, const int *n_near, int cap, int M, const Geo &g,
                 const PotDev &P, float *X, cudaStream_t s, float *mom = nullptr);
void launch_pairgrad(const uint4 *fix, const int *near_keys, const int *n_near, const int *far_keys, const int *n_far,
                     int cap, int cap_far, int M, const Geo &g, const PotDev &P, const float *dEdX, float4 *pair_g,
                     float4 *Fpart, float *E_lj, cudaStream_t s, const float *mom = nullptr);
void launch_force_gather(const int *near_keys, const int *n_near, int cap, int M, int N, int has_mlp,
                         const float4 *pair_g, const float4 *Fpart, const float *E_lj, const float *E_mlp, float *F,
                         float *E_out, DevState *st, cudaStream_t s);
size_t desc_smem_bytes(int warps, int cap);
cudaError_t verify_kernels_setup(int max_smem);

// per-window Verlet candidate lists (lsd_verlet.cu)
struct VerletPlan {
    int nc[3];          // cells per axis (a grid narrower than 3 cells scans all atoms)
    float rlist2f;      // (max cutoff + skin)^2
    float move2f;       // (0.45 skin)^2: largest allowed displacement^2 from the list's base
    int cap, cap_pow2;  // list capacity per atom and its power-of-two sort width
    bool all_pairs;     // grid narrower than 3 cells: every atom is a candidate, no lists are built
};
struct VerletBufs {
    uint4 *fix_base = nullptr;   // [N] fixed point of the base positions
    int *cell_of_atom = nullptr;
    int *cell_count = nullptr;   // [ncells] counts, then fill cursors
    int *cell_start = nullptr;   // [ncells + 1]
    int *cell_atoms = nullptr;   // [N]
    int *cell_scratch = nullptr; // [1] counter of the single-cell case
    int *vlist = nullptr;        // [N][cap] sorted candidate atom indices
    int *vcount = nullptr;       // [N]
};
// skip (device, may be null): nonzero skips the build; rebuild (device, may be
// null): zero skips it (the verdict of launch_verlet_check)
void launch_verlet_build(const VerletPlan &vp, const double *q, const int *species, const Geo &g, VerletBufs &b,
                         DevState *st, cudaStream_t s, const int *skip = nullptr, const int *rebuild = nullptr);
// lists kept across windows: st->list_rebuild = some atom of q lies more than
// sqrt(keep2f) from the lists' base, or st->list_force (then cleared)
void launch_verlet_check(const double *q, const VerletBufs &b, const Geo &g, float keep2f, DevState *st,
                         cudaStream_t s);
cudaError_t verlet_setup(int max_smem);
void launch_neigh_list(const uint4 *fix, const int *vlist, const int *vcount, int vcap, int M, const Geo &g,
                       float rmax2f, float near2f, int cap_near, int cap_far, int *near_keys, int *far_keys,
                       int *n_near, int *n_far, DevState *st, const int *keff, cudaStream_t s, int j_off = 0);

// MLP (lsd_mlp.cu)
void launch_mlp_fp32(const float *X, int M, const PotDev &P, float *E_mlp, float *dEdX, cudaStream_t s);
size_t mlp_fp32_smem_bytes(const PotDev &P);
cudaError_t mlp_kernels_setup(int max_smem);

// MLP on the tcgen05 tensor cores (lsd_mlp_tc.cu): BF16, FP32 as three TF32
// products per term, FP8 e4m3 with static per-tensor scales
enum { kTcBF16 = 0, kTcTF32x3 = 1, kTcFP8 = 2, kTcF16x3 = 3 };
struct TcWeights {
    const void *wn[kMaxLayers][2];   // W_l   [W][din_p] in the operand type; [1] = TF32 lo part
    const void *wt[kMaxLayers][2];   // W_l^T [din_p][W]
};
bool mlp_tc_supported(int op, const PotDev &P);
void *mlp_tc_plan(int op, const PotDev &P, const TcWeights &w);   // tensor maps; nullptr on failure
void mlp_tc_plan_free(void *plan);
int mlp_tc_plan_op(const void *plan);
size_t mlp_tc_smem_bytes(int op);
size_t mlp_tc_scratch_elems(int op, const PotDev &P, int n_cta);   // bf16 SiLU' scratch (0: kept in TMEM)
int mlp_tc_grid(int M, int n_sm);
// scales (FP8 only, device [3L]): A scales of forward GEMMs, of backward GEMMs, weight scales;
// amax (device [2L] or null): |max| of the same A tensors, recorded with atomics (calibration)
void launch_mlp_tc(const void *plan, const float *X, int M, const PotDev &P, float *E_mlp, float *dEdX,
                   __nv_bfloat16 *scratch, const float *scales, float *amax, int n_sm, int *err, cudaStream_t s);
cudaError_t mlp_tc_setup();
size_t mlp_tc_static_scratch_bytes();
int mlp_tc_static_launch(const void *plan, const float *X, int M, const PotDev &P, float *E_mlp, float *dEdX,
                         const float *scales, int n_sm, int *err, cudaStream_t s);

// transport (lsd_transport.cu)
int transport_atoms_per_block(int N);
cudaError_t transport_setup();
// keff: the window's drafted step count (the run state's, or the window
// header's in a pipelined round).  A window verified in stages: K is the end
// of the stage (the decision covers steps 0 .. min(K, k_eff) - 1), j0 its first
// step (steps before it were reduced by earlier stages), staged = 1 for every
// stage but the last, and next the conditional handle of the next stage's
// graph node, set when the window goes on (nothing is committed then).
void launch_transport_reduce(int K, const Geo &g, const Coef &cf, const int *species, const float *Fd,
                             const float *Ft, DevState *st, double2 *partials, const int *keff, cudaStream_t s,
                             int j0 = 0);
void launch_transport_commit(int K, const Geo &g, const Coef &cf, const int *species, const double *w_qmid,
                             const double *w_pdraft, const float *Fd, const float *Ft, const float *Fraw, float *ec_dF,
                             int ec_on, double *q, double *p, double *p_obabo, DevState *st,
                             const double2 *partials, const int *keff, cudaStream_t s, int staged = 0,
                             cudaGraphConditionalHandle next = 0);
void launch_transport(int K, const Geo &g, const Coef &cf, const int *species, const double *w_qmid,
                      const double *w_pdraft, const float *Fd, const float *Ft, const float *Fraw, float *ec_dF,
                      int ec_on, double *q, double *p, double *p_obabo, DevState *st, double2 *partials,
                      const int *keff, cudaStream_t s, int j0 = 0, int staged = 0,
                      cudaGraphConditionalHandle next = 0);

// draft and plain integrator (lsd_draft.cu)
// The grid-form draft's synchronisation words, zeroed before each launch.
struct DraftSync {
    unsigned long long bar;   // grid-barrier arrivals
    unsigned moved;           // K - j of the earliest step j at which an atom left the lists' skin (0: none)
    unsigned abort;           // a CTA's barrier wait ran out of time
};
struct DraftPlan {
    int cluster;      // CTAs in the draft cluster (one per SM); the grid form: CTAs of the cooperative grid
    bool grid;        // the grid form (cooperative launch, grid-wide barriers)
    bool stage_fix;   // positions of a step staged in shared memory
    size_t smem;      // dynamic shared memory per CTA
    bool reg;         // owned atoms' FP64 state in registers
    bool minimg;      // every draft cutoff below 0.499 of every box side: minimum images only
    int noise_steps;  // a launch that drafts at most this many steps draws their noise up front into shared memory
    size_t smem_base; // the shared memory without that noise buffer, and the buffer's bytes per step
    size_t noise_step_bytes;
    size_t max_smem;
    bool stage_list;  // owned atoms' Verlet lists copied to shared memory once per launch
    bool self_list;   // no cell grid: the kernel lists its atoms' candidates itself (in shared memory)
    bool stage_dedx;  // learned draft: every atom's radial dE/dX staged in shared memory each step
    int K;            // window length the plan was made for
    bool ok;
};
DraftPlan draft_plan(int N, int K, const PotDev &P, bool learned, int vcap, bool all_pairs, int max_cluster,
                     size_t max_smem);
constexpr int kGridDraftMinAtoms = 2048;   // smaller systems draft in one cluster only
bool draft_grid_fits(const DraftPlan &pl, bool learned, int n_sm);
DraftPlan draft_grid_plan(int N, int K, const PotDev &P, bool learned, int vcap, bool all_pairs, int n_sm,
                          size_t max_smem);
int draft_max_cluster(size_t smem, bool learned);
// Re-sizes a plan's up-front noise buffer for launches of `steps` drafted steps
// (a window's K, or the stage length of windows verified in stages): the
// buffer holds them when it fits the noise allowance, else it is dropped.
void draft_plan_noise(DraftPlan &pl, int steps);
cudaError_t launch_draft(const DraftPlan &pl, bool learned, int K, const Geo &g, const PotDev &P, const Coef &cf,
                         const VerletPlan &vp, const VerletBufs &vb, const int *species, const double *q,
                         const double *p, const float *ec_dF, int ec_on, DevState *st, double *w_qmid,
                         double *w_pdraft, float *w_Fd, float *w_Fraw, uint4 *w_fix, float *w_dEdX,
                         cudaStream_t s, WinHdr *hdr = nullptr, int redraft = 0, DraftSync *sync = nullptr,
                         int j0 = 0,   // K: the last step + 1 of this launch; j0 > 0 continues a window from step j0
                         // learned draft: per-step neighbour scratch [N][ccap] + counts [N]
                         int *w_nbr = nullptr, int ccap = 0);
// the fused plain-target step (lsd_plain.cu)
constexpr int kPlainMaxN = 512;
struct PlainPlan {
    bool ok;
    bool minimg;      // every cutoff below 0.499 of every box side
    int atoms;        // owned atoms per block (one warp each)
    int blocks;       // cooperative grid: one block per `atoms` atoms
    size_t smem;      // dynamic shared memory per block
    int cap;          // descriptor list capacity (multiple of 32, <= 128)
    int R;            // cap / 32
};
PlainPlan plain_plan(int N, const PotDev &P, bool fp32_target, bool obabo, int cap, const Geo &g, size_t max_smem);
cudaError_t plain_setup(const PlainPlan &pl);
cudaError_t launch_plain_fused(const PlainPlan &pl, int n_steps, const Geo &g, const PotDev &P, const Coef &cf,
                               const int *species, double *q, double *p, uint4 *gfix, int *gkeys, int *gcnt,
                               float4 *gpg, unsigned long long *bar, DevState *st, cudaStream_t s);
// the pipelined window loop (lsd_draft.cu)
void launch_spec_base(const Geo &g, const Coef &cf, const int *species, const double *qmid_b, const double *pdraft_b,
                      const WinHdr *hb, WinHdr *hn, const DevState *st, double *qb, double *pb, cudaStream_t s);
void launch_redraft_flag(DevState *st, WinHdr *hn, cudaStream_t s);
void launch_hdr_invalidate(WinHdr *h, cudaStream_t s);
cudaError_t draft_kernels_setup(int max_smem);
void launch_plain_half(const Geo &g, const Coef &cf, const int *species, const double *q, const double *p,
                       DevState *st, double *qmid, uint4 *fix, cudaStream_t s);
void launch_plain_finish(const Geo &g, const Coef &cf, const int *species, const double *qmid, const float *F,
                         double *q, double *p, double *p_obabo, DevState *st, cudaStream_t s);
void launch_obabo_enter(const Geo &g, const Coef &cf, const int *species, const float *F, long long n, double *p,
                        cudaStream_t s);

}  // namespace lsd
