// lsd_draft.cu -- the serial draft of a window (Alg. 2 draft_step, K times):
//   q_mid = q + (dt/2) p/m                          (A)
//   F~ = draft(q_mid)                               (LJ, or LJ + learned MLP)
//   <p~> = c1 p + (1+c1)(dt/2) kappa (F~ + dF)      (BOB mean, Eq. 4; dF = EC cache)
//   p' = <p~> + sigma xi_n,  q' = q_mid + (dt/2) p'/m  (BOB draw, A)
//
// The K steps are inherently serial; within a step the force evaluation is
// parallel over atoms.  The whole window therefore runs in ONE launch of a
// thread-block cluster (up to 16 CTAs, one per SM): each CTA owns a slice of
// the atoms and writes their half-step fixed-point positions to global memory
// (for the verification) and, when all N fit, into every CTA's shared memory
// by asynchronous stores that complete bytes on the receiving CTA's mbarrier;
// each CTA waits until the step's N positions have landed (bounded wait).
// Larger systems use a cluster barrier and read the positions through L2.
// Large systems also have a grid form of the same kernel: one CTA per SM in a
// cooperative launch, a bounded grid-wide barrier per step in place of the
// cluster barrier, and the displacement flags in global memory.  The per-atom
// arithmetic (and its order) is the cluster form's, so both give the same
// bits; the window loop runs the grid form when nothing else needs the SMs
// (an unpipelined window, a redraft) and the cluster form for the speculative
// draft that overlaps a verification.
//
// Candidates come from Verlet lists (cutoff + skin around a base): the
// window's lists from lsd_verlet.cu on a cell grid of three or more cells per
// axis, else lists each CTA builds for its own atoms at launch from one scan
// over all atoms (no cell grid).  At every step each CTA checks its atoms'
// displacement from the base; if any atom moved more than 0.45 skin the whole
// cluster stops drafting at that step (k_eff < K, decided identically in every
// CTA from the exchanged flags), because the lists are no longer guaranteed
// complete.  Each list entry is tested with the exact membership rule, so the
// interacting set is the rule's set, not an approximation.  When neither kind
// of list fits in shared memory every atom is a candidate: no lists, no
// displacement check, k_eff = K.
//
// FP64 only for the state updates, with explicit round-to-nearest intrinsics
// so the half-step positions are reproducible bit for bit.
#include "lsd_common.cuh"
#include "lsd_kernels.h"
#include "lsd_tc.cuh"

namespace lsd {

constexpr int kDraftThreads = 512;
constexpr int kDraftWarps = kDraftThreads / 32;
constexpr int kSegCap = 128;       // staged descriptor neighbours per species per warp (learned draft)
constexpr int kLearnW = 32;        // the learned draft's hidden units (one layer, one unit per lane)
// floats of one warp's learned-draft stage ([S][2][kSegCap] + the input vector) and of the CTA's weight copies
__host__ __device__ inline int learned_stage_floats(int S, int d0p) { return 2 * S * kSegCap + d0p; }
__host__ __device__ inline int learned_weight_floats(int d0p) { return 2 * kLearnW * d0p + kLearnW; }
constexpr int kMaxCluster = 16;    // largest draft cluster

__device__ __forceinline__ void cluster_barrier() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

// A barrier over every CTA of a cooperative launch (one CTA per SM, all
// resident).  Bounded: it gives up after about two seconds, or at once when
// another CTA has given up (sync->abort), so a stalled grid ends within one
// time-out instead of one per remaining step.
// (No static shared memory: the kernels' dynamic allowance is the device's maximum.)
__device__ bool draft_grid_barrier(DraftSync *sync, unsigned total) {
    int ok = 1;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned long long arrive = atomicAdd(&sync->bar, 1ull);
        const unsigned long long target = (arrive / total + 1ull) * total;
        const long long t0 = clock64();
        for (;;) {
            unsigned long long v;
            unsigned ab;
            asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(&sync->bar) : "memory");
            if (v >= target) break;
            asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(ab) : "l"(&sync->abort) : "memory");
            if (ab != 0u || clock64() - t0 > 4000000000ll) {
                ok = 0;
                atomicExch(&sync->abort, 1u);
                break;
            }
        }
        __threadfence();
    }
    return __syncthreads_and(ok) != 0;   // thread 0's verdict, for every thread
}


// Positions of window step j: staged in shared memory when they fit, else read
// through L2 (ld.global.cg: other CTAs of the cluster wrote them this launch).
struct FixView {
    const uint4 *smem;
    const uint4 *glob;
    __device__ __forceinline__ uint4 operator[](int k) const { return smem ? smem[k] : __ldcg(glob + k); }
};

// The candidate list of an owned atom: its copy in shared memory (staged once
// per launch) or the global Verlet list.
struct ListView {
    const int *p;
    bool smem;
    __device__ __forceinline__ int operator[](int t) const { return smem ? p[t] : __ldg(p + t); }
};

// Every image of atom k that passes the per-axis bound around atom i, as
// fn(dx, dy, dz, d2).  With minimg (every cutoff below 0.499 of every box side)
// only the minimum image can lie within the cutoff: the other image along an
// axis is at least L/2 (less rounding) away, so the rule's set is the set of
// minimum images that pass d2 < rc2, and the general enumeration is skipped.
template <class Fn>
__device__ __forceinline__ void for_images(const Geo &g, uint4 fi, uint4 fk, float rc2, bool minimg, Fn &&fn) {
    if (minimg) {
        float dx, dy, dz;
        int kk;
        axis_min(fi.x, fk.x, g.scale_f[0], dx, kk);
        axis_min(fi.y, fk.y, g.scale_f[1], dy, kk);
        axis_min(fi.z, fk.z, g.scale_f[2], dz, kk);
        fn(dx, dy, dz, dist2_rule(dx, dy, dz));
        return;
    }
    const AxisOpts ox = axis_opts(fi.x, fk.x, g.scale_f[0], g.Lf[0], rc2);
    const AxisOpts oy = axis_opts(fi.y, fk.y, g.scale_f[1], g.Lf[1], rc2);
    const AxisOpts oz = axis_opts(fi.z, fk.z, g.scale_f[2], g.Lf[2], rc2);
    for (int bz = 0; bz < oz.n; ++bz)
        for (int by = 0; by < oy.n; ++by)
            for (int bx = 0; bx < ox.n; ++bx) {
                const float dx = opt_d(ox, bx), dy = opt_d(oy, by), dz = opt_d(oz, bz);
                fn(dx, dy, dz, dist2_rule(dx, dy, dz));
            }
}

// The draft's cutoff function, fc = (1 + cos(pi r / rc)) / 2 and its
// derivative, from r and 1/rc (the target's descriptors divide by rc).
__device__ __forceinline__ void draft_cutoff(float r, float inv_rc, float &fc, float &dfc) {
    float sn, cs;
    sincospif(r * inv_rc, &sn, &cs);
    fc = 0.5f * (cs + 1.0f);
    dfc = (-0.5f * 3.14159265358979f) * inv_rc * sn;
}

// Learned draft, first phase: radial descriptors of atom i from its candidate
// list (all atoms when cand is null), the MLP (BF16 operands, FP32
// accumulation), dE/dx written to g_out[d0p].  The warp's stage holds, per
// species s, the (r, fc) of the atom's neighbours of species s in list order
// ([S][2][kSegCap]), so the basis sums run over one species at a time; xbuf
// holds the BF16-rounded input vector.  wf / wtf / wo: FP32 copies of the BF16
// first layer ([W][d0p] and [d0p][W], W = 32 hidden units, one per lane) and
// output weights, staged once per launch.  Returns false when some species
// had more than kSegCap neighbours (its sum is then truncated).
__device__ bool learned_atom_grad(const PotDev &P, const Geo &g, const FixView &fx, int i, const ListView cand, int nc,
                                  bool minimg, float inv_rc, float rc2_all, float *stage, float *xbuf,
                                  const float *wf, const float *wtf, const float *wo, float *g_out, int *nbr_row,
                                  int *nbr_count, int ccap) {
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const uint4 fi = fx[i];
    const int S = g.S;
    int cnt[kMaxSpecies];
#pragma unroll
    for (int s = 0; s < kMaxSpecies; ++s) cnt[s] = 0;
    int nn = 0;   // candidates with an image within the draft's largest cutoff, in list order (the second phase's)
    // candidates four per lane in flight: their list entries and positions are loaded before any is tested
    constexpr int kB = 4;
    for (int base0 = 0; base0 < nc; base0 += 32 * kB) {
        int kq[kB];
        uint4 fq[kB];
#pragma unroll
        for (int u = 0; u < kB; ++u) {
            const int t = base0 + 32 * u + lane;
            kq[u] = t < nc ? (cand.p ? cand[t] : t) : i;
        }
#pragma unroll
        for (int u = 0; u < kB; ++u) fq[u] = kq[u] != i ? fx[kq[u]] : fi;
#pragma unroll
        for (int u = 0; u < kB; ++u) {
            if (base0 + 32 * u >= nc) break;   // uniform over the warp
            const int k = kq[u];
            const uint4 fk = fq[u];
            const int sk = (int)fk.w;
            bool any = false;   // some image of k within rc_all
            if (minimg) {
                // at most one image within the cutoff: each species' neighbours placed by one ballot
                bool in = false;
                float r = 0.f;
                if (k != i) {
                    float dx, dy, dz;
                    int kk;
                    axis_min(fi.x, fk.x, g.scale_f[0], dx, kk);
                    axis_min(fi.y, fk.y, g.scale_f[1], dy, kk);
                    axis_min(fi.z, fk.z, g.scale_f[2], dz, kk);
                    const float d2 = dist2_rule(dx, dy, dz);
                    any = d2 < rc2_all;
                    in = d2 < P.desc_rc2f;
                    if (in) r = d2 * rsqrtf(d2);
                }
#pragma unroll
                for (int s = 0; s < kMaxSpecies; ++s) {
                    if (s >= S) break;
                    const bool mine = in && sk == s;
                    const unsigned m = __ballot_sync(0xffffffffu, mine);
                    const int w = cnt[s] + __popc(m & lt);
                    if (mine && w < kSegCap) stage[(2 * s) * kSegCap + w] = r;
                    cnt[s] += __popc(m);
                }
            } else {
                // the (at most 8) images of k within the descriptor cutoff, in enumeration order
                float rs[8];
                int nm = 0;
                if (k != i)
                    for_images(g, fi, fk, rc2_all, false, [&](float, float, float, float d2) {
                        any = any || d2 < rc2_all;
                        if (d2 < P.desc_rc2f && nm < 8) rs[nm++] = d2 * rsqrtf(d2);
                    });
#pragma unroll
                for (int s = 0; s < kMaxSpecies; ++s) {
                    if (s >= S) break;
                    const int mine = (k != i && sk == s) ? nm : 0;
                    int sc = mine;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const int v = __shfl_up_sync(0xffffffffu, sc, o);
                        if (lane >= o) sc += v;
                    }
                    int w = cnt[s] + sc - mine;
                    for (int c = 0; c < mine; ++c, ++w)
                        if (w < kSegCap) stage[(2 * s) * kSegCap + w] = rs[c];
                    cnt[s] += __shfl_sync(0xffffffffu, sc, 31);
                }
            }
            const unsigned ma = __ballot_sync(0xffffffffu, any);
            const int wn = nn + __popc(ma & lt);
            if (any && wn < ccap) nbr_row[wn] = k;
            nn += __popc(ma);
        }
    }
    if (lane == 0) *nbr_count = nn < ccap ? nn : ccap;
    const int nr = P.n_rbf;
    for (int f = lane; f < P.d0p; f += 32) xbuf[f] = 0.f;
    __syncwarp();
    // the cutoff function of every staged neighbour, lanes over neighbours (in the scan above most lanes of a
    // candidate chunk lie outside the cutoff)
#pragma unroll
    for (int s = 0; s < kMaxSpecies; ++s) {
        if (s >= S) break;
        const int n = cnt[s] < kSegCap ? cnt[s] : kSegCap;
        for (int p = lane; p < n; p += 32) {
            float fc, dfc;
            draft_cutoff(stage[(2 * s) * kSegCap + p], inv_rc, fc, dfc);
            stage[(2 * s + 1) * kSegCap + p] = fc;
        }
    }
    __syncwarp();
    bool ok = nn <= ccap;
    {
        // lanes over basis functions (8 or 16 wide), the groups of lanes over one species' neighbours, then a
        // reduction over the groups: every lane busy for n_rbf <= 8 as for 16
        const int nb = nr <= 8 ? 8 : 16;
        const int kb = lane & (nb - 1), ng = 32 / nb;
        const float mu = (float)kb * P.rbf_w;
#pragma unroll
        for (int s = 0; s < kMaxSpecies; ++s) {
            if (s >= S) break;
            ok = ok && cnt[s] <= kSegCap;
            const int n = cnt[s] < kSegCap ? cnt[s] : kSegCap;
            const float *sr = stage + (2 * s) * kSegCap, *sfc = sr + kSegCap;
            float acc = 0.f;
            if (kb < nr)
                for (int p = lane / nb; p < n; p += ng) {
                    const float t = sr[p] - mu;
                    acc += __expf(-t * t * P.rbf_inv2w2) * sfc[p];   // the hardware exponential, as the target's basis
                }
            for (int o = 16; o >= nb; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
            if (lane < nr) xbuf[s * nr + lane] = __bfloat162float(__float2bfloat16(acc));
        }
        if (lane == 0) xbuf[S * nr + P.n_ang + (int)fi.w] = 1.f;
    }
    __syncwarp();
    // one hidden unit per lane (W = 32): h = b + W x, dE/dh = w_out SiLU'(h) (linear head: dE/dy = 1)
    float h = P.b[0][lane];
    for (int f = 0; f < P.d0; ++f) h = fmaf(wtf[f * kLearnW + lane], xbuf[f], h);
    const float gh = wo[lane] * dsiluf_(h);
    // dE/dx_f = sum_u W[u][f] gh_u: lane f over the hidden units, gh_u handed round by shuffles
    for (int f0 = 0; f0 < P.d0p; f0 += 32) {
        const int f = f0 + lane;
        float v = 0.f;
        for (int u = 0; u < kLearnW; ++u) {
            const float gu = __shfl_sync(0xffffffffu, gh, u);
            if (f < P.d0) v = fmaf(wf[u * P.d0p + f], gu, v);
        }
        if (f < P.d0p) g_out[f] = v;
    }
    __syncwarp();
    return ok;
}

// Store v at the same shared-memory offset as `local` in CTA `rank` of the cluster.
__device__ __forceinline__ void st_cluster(const void *local, uint32_t rank, uint4 v) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(local);
    uint32_t ra;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(rank));
    asm volatile("st.shared::cluster.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(ra), "r"(v.x), "r"(v.y), "r"(v.z),
                 "r"(v.w)
                 : "memory");
}
__device__ __forceinline__ void st_cluster(const int *local, uint32_t rank, int v) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(local);
    uint32_t ra;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(rank));
    asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(ra), "r"(v) : "memory");
}

// One launch drafts the whole window.  Per step:
//   A  half-step positions of owned atoms (FP64, one lane per coordinate, four
//      lanes per atom), their fixed point written to global memory for the
//      verification and, when the positions fit in shared memory, stored
//      directly into every CTA's copy (asynchronous distributed-shared-memory
//      stores, double-buffered by step parity, each completing bytes on the
//      receiving CTA's mbarrier of that parity); with Verlet lists, each CTA's
//      displacement flag, stored into its own slot in every CTA the same way
//   B  wait until all N positions (and C flags) of the step have landed in this
//      CTA -- no cluster-wide barrier, so no fence waits for this step's global
//      stores; a CTA reaches step j+2 (which rewrites the buffers of step j)
//      only after every CTA sent step j+1, which each does after reading step
//      j.  Without staged positions: a cluster barrier, positions from global
//      memory.  Stop when any CTA flagged a displacement
//   C  forces on owned atoms (one warp per atom, lanes over the candidates:
//      the atom's Verlet list, or all atoms when vlist is null)
//   D  BOB + A, one lane per coordinate
// REG keeps owned atoms' FP64 state in registers (a CTA owns at most
// kRegPasses * kGroups atoms); otherwise it is re-read from the window arrays.
constexpr int kGroups = kDraftThreads / 4;   // four-lane groups: one atom, lanes 0..2 its coordinates
constexpr int kRegPasses = 2;

// Valid iff the speculative base is the committed state: the previous window
// committed up to the base step without a rejection (a rejection at its last
// step also ends at that step index, but in the reflected state).
__device__ __forceinline__ bool spec_is_valid(const WinHdr *hn, const DevState *st) {
    return hn->skip == 0 && hn->base == st->step && st->first_reject_last == -1;
}

// GRID: the grid form (gridDim.x CTAs of a cooperative launch; stage_fix and
// self_list are 0; sync zeroed before the launch).
template <bool LEARNED, bool REG, bool GRID>
__global__ void __launch_bounds__(kDraftThreads, 1)
    draft_window_cluster_kernel(int K, Geo g, PotDev P, Coef cf, const int *__restrict__ vlist,
                                const int *__restrict__ vcount, int vcap, const uint4 *__restrict__ fix_base,
                                float move2f, float rlist2f, int stage_fix, int minimg, int noise_smem,
                                int stage_list, int self_list, int stage_dedx,
                                const int *__restrict__ species,
                                const double *__restrict__ q_base, const double *__restrict__ p_base,
                                const float *__restrict__ ec_dF, int ec_on, DevState *__restrict__ st,
                                double *__restrict__ w_qmid, double *__restrict__ w_pdraft, float *__restrict__ w_Fd,
                                float *__restrict__ w_Fraw, uint4 *__restrict__ w_fix, float *__restrict__ w_dEdX,
                                int *__restrict__ w_nbr, int ccap,
                                WinHdr *__restrict__ hdr, int redraft, DraftSync *__restrict__ sync, int j0) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int N = g.N;
    const int C = gridDim.x, c = blockIdx.x;
    const int A = (N + C - 1) / C;           // owned atoms per CTA
    const int a0 = c * A, a1 = min(N, a0 + A);
    const int nown = a1 > a0 ? a1 - a0 : 0;
    const bool use_list = vlist != nullptr || self_list;
    float4 *sF = (float4 *)smraw;                               // [A]
    uint4 *sbase = (uint4 *)(sF + A);                           // [A] list base positions of owned atoms (lists)
    float *slj = (float *)(sbase + (use_list ? A : 0));         // sig2, eps24 tables
    float *sstage = slj + 2 * kMaxSpecies * kMaxSpecies;        // learned: per warp [S][2][kSegCap] + d0p
    const int stage_stride = learned_stage_floats(g.S, P.d0p);
    float *swf = sstage + (LEARNED ? (size_t)kDraftWarps * stage_stride : 0);   // learned: W1 [W][d0p], FP32
    float *swtf = swf + kLearnW * P.d0p;                                         //          W1^T [d0p][W]
    float *swo = swtf + kLearnW * P.d0p;                                         //          w_out [W]
    uint4 *sfix = (uint4 *)(swf + (LEARNED ? learned_weight_floats(P.d0p) : 0));  // [2][N]
    // displacement flags: [2] (cluster-barrier exchange) or [2][kMaxCluster], one slot per sending CTA
    int *sflag = (int *)(sfix + (stage_fix ? 2 * (size_t)N : 0));
    // [3] mbarriers: the two exchange barriers (staged positions, by step parity) and the exit barrier of a
    // window that gave up waiting
    uint64_t *sbar = (uint64_t *)(sflag + 2 * kMaxCluster);
    float *snoise = (float *)(sbar + 3);   // [K - j0][A][3] when noise_smem: the launch's xi, drawn up front
    // Read-only per-atom data of owned atoms, staged once: a cluster barrier's
    // acquire leaves no global line in L1, so a per-step global read is an L2
    // round trip on the step's critical path.
    int *sspec = (int *)(snoise + (noise_smem ? (size_t)(K - j0) * A * 3 : 0));   // [A] species
    int *svc = sspec + A;                                                  // [A] list lengths (stage_list)
    int *svl = svc + A;                                                    // [A][vcap] lists (stage_list)
    // learned draft, small systems: the radial dE/dX of every atom, [N][S n_rbf], staged once per step
    float *sdedx = (float *)(sspec + A + (stage_list ? (size_t)A * (vcap + 1) : 0));
    // the base step: the committed one, or (pipelined loop) the window header's;
    // a redraft runs only when the speculative draft of this window does not
    // stand, from the committed state.  Uniform over the cluster: the header is
    // rewritten only after the last cluster barrier.
    long long n0;
    if (hdr && redraft) {
        if (spec_is_valid(hdr, st) || st->step >= st->target_step) return;
        n0 = st->step;
    } else if (hdr) {
        if (hdr->skip || hdr->base >= st->target_step) return;
        n0 = hdr->base;
    } else {
        if (st->step >= st->target_step) return;
        n0 = st->step;
    }
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int grp = tid >> 2, x = tid & 3, gl = lane & ~3;
    const size_t D = (size_t)3 * N;
    const int passes = (nown + kGroups - 1) / kGroups;
    constexpr int kP = REG ? kRegPasses : 1;
    const float rc2_all = LEARNED ? fmaxf(P.lj_rc2f, P.desc_rc2f) : P.lj_rc2f;
    const double scale_x = x == 0 ? g.scale[0] : (x == 1 ? g.scale[1] : g.scale[2]);
    for (int t = tid; t < g.S * g.S; t += blockDim.x) {
        slj[t] = P.lj_sig2[t];
        slj[kMaxSpecies * kMaxSpecies + t] = P.lj_eps24[t];
    }
    // the learned draft's single hidden layer, read by every atom of every step: FP32 copies of its BF16 values
    const float inv_rc = LEARNED ? 1.f / P.desc_rc : 0.f;
    if (LEARNED) {
        for (int t = tid; t < kLearnW * P.d0p; t += blockDim.x) {
            swf[t] = __bfloat162float(P.Wn_bf[0][t]);
            swtf[t] = __bfloat162float(P.Wt_bf[0][t]);
        }
        if (tid < kLearnW) swo[tid] = __bfloat162float(P.wout_bf[tid]);
    }
    if (tid < 2 * kMaxCluster) sflag[tid] = 0;
    const uint32_t bar0 = tc::smem_u32(sbar);
    if (stage_fix && tid == 0) {
        tc::mbar_init(bar0, 1);
        tc::mbar_init(bar0 + 8, 1);
        tc::mbar_init(bar0 + 16, C);
        tc::mbar_fence_init();
    }
    // bytes that land in this CTA per step: every atom's position, every CTA's flag
    const uint32_t step_bytes = (uint32_t)(N * sizeof(uint4) + (use_list ? C * sizeof(int) : 0));
    // remote bases of the CTAs this lane sends positions to (ranks x, x+4, x+8, x+12)
    uint32_t rfix[4], rbar[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const int r = x + 4 * m;
        rfix[m] = rbar[m] = 0u;
        if (stage_fix && r < C) {
            rfix[m] = tc::cluster_map(tc::smem_u32(sfix), (uint32_t)r);
            rbar[m] = tc::cluster_map(bar0, (uint32_t)r);
        }
    }
    for (int ii = tid; ii < nown; ii += blockDim.x) {
        sspec[ii] = species[a0 + ii];
        if (vlist) sbase[ii] = fix_base[a0 + ii];
        if (vlist && stage_list) svc[ii] = vcount[a0 + ii];
    }
    if (vlist && stage_list)
        for (int e = tid; e < nown * vcap; e += blockDim.x) {
            const int ii = e / vcap, t = e - ii * vcap;
            if (t < vcount[a0 + ii]) svl[e] = vlist[(size_t)(a0 + ii) * vcap + t];
        }
    if (self_list) {
        // No cell grid (box narrower than three list radii): each CTA lists its
        // own atoms' candidates itself, by one scan over every atom's base
        // position (minimum images: if any image of k lies within the list
        // radius, the minimum one does), in index order.  The base positions
        // of all atoms go to the step-1 position buffer, which other CTAs
        // first write after this CTA has sent its step-0 positions.
        uint4 *sb_all = sfix + N;
        for (int k = tid; k < N; k += blockDim.x)
            sb_all[k] = make_uint4(fixpoint(q_base[3 * k], g.scale[0]), fixpoint(q_base[3 * k + 1], g.scale[1]),
                                   fixpoint(q_base[3 * k + 2], g.scale[2]), (unsigned)species[k]);
        __syncthreads();
        for (int ii = warp; ii < nown; ii += kDraftWarps) {
            const int i = a0 + ii;
            const uint4 fi = sb_all[i];
            int cnt = 0;
            for (int b0 = 0; b0 < N; b0 += 32) {
                const int k = b0 + lane;
                bool in = false;
                if (k < N && k != i) {
                    const uint4 fk = sb_all[k];
                    float dx, dy, dz;
                    int kk;
                    axis_min(fi.x, fk.x, g.scale_f[0], dx, kk);
                    axis_min(fi.y, fk.y, g.scale_f[1], dy, kk);
                    axis_min(fi.z, fk.z, g.scale_f[2], dz, kk);
                    in = dist2_rule(dx, dy, dz) < rlist2f;
                }
                const unsigned bal = __ballot_sync(0xffffffffu, in);
                const int pos = cnt + __popc(bal & ((1u << lane) - 1u));
                if (in && pos < vcap) svl[(size_t)ii * vcap + pos] = k;
                cnt += __popc(bal);
            }
            if (lane == 0) {
                sbase[ii] = fi;
                svc[ii] = cnt < vcap ? cnt : vcap;
                if (cnt > vcap) atomicOr(&st->err, 1);
            }
        }
        __syncthreads();
    }
    // REG: coordinate x of owned atoms grp + p * kGroups
    // (and the atom's per-species constants: the half-step drift factor and sigma)
    double qr[kP], pr[kP], hmr[kP], sgr[kP];
    float dfr[kP], xr[kP];
#pragma unroll
    for (int p = 0; p < kP; ++p) {
        qr[p] = pr[p] = hmr[p] = sgr[p] = 0.0;
        dfr[p] = xr[p] = 0.f;
        const int ii = grp + p * kGroups;
        if (REG && ii < nown && x < 3) {
            const int i = a0 + ii;
            const int sp = species[i];
            // a launch that continues a window (j0 > 0) starts from the last drafted step's state
            qr[p] = j0 == 0 ? q_base[3 * i + x] : w_qmid[(size_t)(j0 - 1) * D + 3 * i + x];
            pr[p] = j0 == 0 ? p_base[3 * i + x] : w_pdraft[(size_t)(j0 - 1) * D + 3 * i + x];
            dfr[p] = ec_on ? ec_dF[3 * i + x] : 0.f;
            hmr[p] = cf.obabo ? species_pick(cf.hmf, sp) : species_pick(cf.hm, sp);
            sgr[p] = species_pick(cf.sig, sp);
        }
    }
    // threads of the last warp (idle while warps 0-1 run the FP64 updates) post
    // each step's expected bytes and send this CTA's displacement flag
    const int side = tid - (int)(blockDim.x - 32);
    // the noise of every step of the window, when it fits: off the per-step critical path
    if (noise_smem) {
        for (int idx = tid; idx < (K - j0) * nown; idx += blockDim.x) {
            const int jl = idx / nown, ii = idx - jl * nown;
            const float3 xi = normals3(cf.seed, (unsigned long long)(n0 + j0 + jl + 1), (uint32_t)(a0 + ii), 0u);
            float *o = snoise + ((size_t)jl * A + ii) * 3;
            o[0] = xi.x;
            o[1] = xi.y;
            o[2] = xi.z;
        }
    }
    // every CTA has started, zeroed its flags and initialised its mbarriers before the first remote store
    if (!GRID && (stage_fix || use_list)) cluster_barrier();
    __syncthreads();
    int keff = K;
    bool gave_up = false;   // this CTA's wait for a step's positions ran out of time
    for (int j = j0; j < K; ++j) {
        const int jl = j - j0;   // the launch's own step count: buffer parity, barrier phases, staged noise
        const int par = jl & 1;
        const unsigned long long n = (unsigned long long)(n0 + j + 1);
        if (stage_fix && side == 31) tc::mbar_expect_tx(bar0 + 8 * par, step_bytes);
        // A: half-step positions, fixed point, broadcast, displacement from the list's base
        int moved = 0;
        // c1 p and sigma xi of this step's BOB (force-independent, the same roundings as in D):
        // with the noise staged, formed in A right after the drift, under its latency
        double c1p[kP], sxi[kP];
#pragma unroll
        for (int p = 0; p < kP; ++p) c1p[p] = sxi[p] = 0.0;
        auto step_a = [&](int p, double &qreg, double &preg) {
            const int ii = grp + p * kGroups;
            const bool own = ii < nown;
            const int i = a0 + (own ? ii : 0);
            const int sp = own ? sspec[ii] : 0;
            uint32_t u = 0u;
            if (own && x < 3) {
                // ABOBA: trailing A of the previous step, then A; staggered OBABO: one full-step A
                const double hm = REG ? hmr[p] : (cf.obabo ? species_pick(cf.hmf, sp) : species_pick(cf.hm, sp));
                double qv, pv;
                if (REG) {
                    pv = preg;
                    qv = (j == 0 || cf.obabo) ? qreg : __dadd_rn(qreg, __dmul_rn(pv, hm));
                } else if (j == 0) {
                    qv = q_base[3 * i + x];
                    pv = p_base[3 * i + x];
                } else {
                    const size_t o = (size_t)(j - 1) * D + 3 * i + x;
                    pv = w_pdraft[o];
                    qv = cf.obabo ? w_qmid[o] : __dadd_rn(w_qmid[o], __dmul_rn(pv, hm));
                }
                const double qm = __dadd_rn(qv, __dmul_rn(pv, hm));
                if (REG) qreg = qm;
                w_qmid[(size_t)j * D + 3 * i + x] = qm;
                u = fixpoint(qm, scale_x);
                // after the conversion the exchange waits for, so they queue behind it on the FP64 pipe
                if (REG && noise_smem) {
                    c1p[p] = __dmul_rn(cf.c1, pv);
                    sxi[p] = __dmul_rn(sgr[p], (double)snoise[((size_t)jl * A + ii) * 3 + x]);
                }
            }
            const uint32_t ux = __shfl_sync(0xffffffffu, u, gl), uy = __shfl_sync(0xffffffffu, u, gl + 1),
                           uz = __shfl_sync(0xffffffffu, u, gl + 2);
            if (own) {
                const uint4 fv = make_uint4(ux, uy, uz, (unsigned)sp);
                if (x == 0) w_fix[(size_t)j * N + i] = fv;
                if (stage_fix) {
                    const uint32_t off = (uint32_t)(((size_t)par * N + i) * sizeof(uint4));
#pragma unroll
                    for (int m = 0; m < 4; ++m)
                        if (x + 4 * m < C) tc::st_async(rfix[m] + off, fv, rbar[m] + 8 * par);
                }
                if (use_list && x == 0) {
                    const uint4 b = sbase[ii];
                    float dmin, d2;
                    int kk;
                    axis_min(b.x, ux, g.scale_f[0], dmin, kk);
                    d2 = dmin * dmin;
                    axis_min(b.y, uy, g.scale_f[1], dmin, kk);
                    d2 += dmin * dmin;
                    axis_min(b.z, uz, g.scale_f[2], dmin, kk);
                    d2 += dmin * dmin;
                    moved |= d2 > move2f;
                }
            }
        };
        if (REG) {
#pragma unroll
            for (int p = 0; p < kP; ++p)
                if (p < passes) step_a(p, qr[p], pr[p]);
        } else {
            double dq, dp;
            for (int p = 0; p < passes; ++p) step_a(p, dq, dp);
        }
        if (use_list) {
            moved = __syncthreads_or(moved);
            if (GRID) {
                // K - j: the largest value marks the earliest step at which an atom left the skin
                if (moved && tid == 0) atomicMax(&sync->moved, (unsigned)(K - j));
            } else if (stage_fix) {
                if (side >= 0 && side < C)
                    tc::st_async(tc::cluster_map(tc::smem_u32(sflag + par * kMaxCluster + c), (uint32_t)side),
                                 moved ? 1u : 0u, tc::cluster_map(bar0 + 8 * par, (uint32_t)side));
            } else if (moved && tid < C) {
                st_cluster(sflag + par, (uint32_t)tid, 1);
            }
        }
        // noise of this step's B, independent of the positions: drawn while the barrier completes
        if (REG && !noise_smem) {
#pragma unroll
            for (int p = 0; p < kP; ++p) {
                const int ii = grp + p * kGroups;
                if (p < passes && ii < nown && x < 3) {
                    const float3 xi = normals3(cf.seed, n, (uint32_t)(a0 + ii), 0u);
                    xr[p] = x == 0 ? xi.x : (x == 1 ? xi.y : xi.z);
                }
            }
        }
        // without staged noise, the products are formed here, once xi is drawn
        if (REG && !noise_smem) {
#pragma unroll
            for (int p = 0; p < kP; ++p) {
                const int ii = grp + p * kGroups;
                if (p < passes && ii < nown && x < 3) {
                    c1p[p] = __dmul_rn(cf.c1, pr[p]);
                    sxi[p] = __dmul_rn(sgr[p], (double)xr[p]);
                }
            }
        }
        // B: this step's positions and flags in this CTA; stop drafting when any
        // atom left the skin (the same flags in every CTA)
        if (stage_fix) {
            const bool ok = tc::mbar_wait_cluster(bar0 + 8 * par, (uint32_t)((jl >> 1) & 1));
            const int f = (use_list && lane < C) ? sflag[par * kMaxCluster + lane] : 0;
            const int code = __syncthreads_or((ok ? 0 : 2) | (f ? 1 : 0));
            if (code) {
                if ((code & 2) && tid == 0) atomicOr(&st->err, 8);
                gave_up = (code & 2) != 0;
                keff = j;
                break;
            }
        } else if (GRID) {
            if (!draft_grid_barrier(sync, (unsigned)C)) {
                if (tid == 0) atomicOr(&st->err, 8);
                keff = j;
                break;
            }
            // every flag of steps <= j was raised before this barrier; later steps' flags are smaller
            if (use_list && *(volatile unsigned *)&sync->moved >= (unsigned)(K - j)) {
                keff = j;
                break;
            }
        } else {
            cluster_barrier();
            if (use_list && sflag[par]) {
                keff = j;
                break;
            }
        }
        FixView fx{stage_fix ? sfix + (size_t)par * N : nullptr, w_fix + (size_t)j * N};
        if (LEARNED) {
            float *stage = sstage + (size_t)warp * stage_stride;
            bool all_in = true;
            for (int ii = warp; ii < nown; ii += kDraftWarps) {
                const int i = a0 + ii;
                const ListView cand{use_list ? (stage_list ? svl + (size_t)ii * vcap : vlist + (size_t)i * vcap)
                                             : nullptr,
                                    stage_list != 0};
                all_in &= learned_atom_grad(P, g, fx, i, cand, use_list ? (stage_list ? svc[ii] : vcount[i]) : N,
                                            minimg != 0, inv_rc, rc2_all, stage, stage + 2 * g.S * kSegCap, swf, swtf,
                                            swo, w_dEdX + (size_t)i * P.d0p, w_nbr + (size_t)i * ccap,
                                            w_nbr + (size_t)N * ccap + i, ccap);
            }
            if (!all_in && lane == 0) atomicOr(&st->err, 1);   // a species' staged neighbours overflowed
            // dE/dx of every atom visible to every CTA
            if (GRID) {
                if (!draft_grid_barrier(sync, (unsigned)C)) {
                    if (tid == 0) atomicOr(&st->err, 8);
                    keff = j;
                    break;
                }
            } else {
                cluster_barrier();
            }
            if (stage_dedx) {
                // the radial block of every atom's dE/dX into shared memory: one coalesced pass
                // instead of two L2 round trips per neighbour pair and basis function
                const int SR = g.S * P.n_rbf;
                for (int e = tid; e < N * SR; e += blockDim.x)
                    sdedx[e] = __ldcg(w_dEdX + (size_t)(e / SR) * P.d0p + (e % SR));
                __syncthreads();
            }
        }
        // C: forces on owned atoms, one warp per atom, lanes over its candidates
        for (int ii = warp; ii < nown; ii += kDraftWarps) {
            const int i = a0 + ii;
            const uint4 fi = fx[i];
            const int si = (int)fi.w;
            const ListView lst{use_list ? (stage_list ? svl + (size_t)ii * vcap : vlist + (size_t)i * vcap) : nullptr,
                               stage_list != 0};
            const int nl = use_list ? (stage_list ? svc[ii] : vcount[i]) : N;
            float fxx = 0.f, fyy = 0.f, fzz = 0.f;
            if (!LEARNED && minimg) {
                // pair-only draft, minimum images: four independent candidates per
                // lane in flight (loads first, then arithmetic), LJ by predication;
                // compiled once per way of reaching positions and candidates, so the
                // staged case reads shared memory with no per-load selection
                auto gather = [&](auto pos_at, auto cand_at) {
                    for (int t0 = lane; t0 < nl; t0 += 128) {
                        uint4 fk[4];
                        int kk[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const int t = t0 + 32 * u;
                            kk[u] = t < nl ? cand_at(t) : i;
                            fk[u] = pos_at(kk[u]);
                        }
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            float dx, dy, dz;
                            int kx;
                            axis_min(fi.x, fk[u].x, g.scale_f[0], dx, kx);
                            axis_min(fi.y, fk[u].y, g.scale_f[1], dy, kx);
                            axis_min(fi.z, fk[u].z, g.scale_f[2], dz, kx);
                            const float d2 = dist2_rule(dx, dy, dz);
                            const bool in = kk[u] != i && d2 < P.lj_rc2f;
                            const int pr2 = si * g.S + (int)fk[u].w;
                            const float sig2 = slj[pr2], eps24 = slj[kMaxSpecies * kMaxSpecies + pr2];
                            const float inv = __fdividef(1.f, in ? d2 : 1.f);
                            const float s2 = sig2 * inv;
                            const float s6 = s2 * s2 * s2, s12 = s6 * s6;
                            const float fr = in ? -eps24 * (2.f * s12 - s6) * inv : 0.f;
                            fxx += fr * dx;
                            fyy += fr * dy;
                            fzz += fr * dz;
                        }
                    }
                };
                if (stage_fix && use_list && stage_list) {
                    const uint4 *sp = sfix + (size_t)par * N;
                    const int *sl = svl + (size_t)ii * vcap;
                    gather([&](int k) { return sp[k]; }, [&](int t) { return sl[t]; });
                } else if (stage_fix && !use_list) {
                    const uint4 *sp = sfix + (size_t)par * N;
                    gather([&](int k) { return sp[k]; }, [&](int t) { return t; });
                } else {
                    gather([&](int k) { return fx[k]; }, [&](int t) { return use_list ? lst[t] : t; });
                }
            }
            // (the learned draft, or general images) candidates four per lane in flight, each lane's in list order;
            // the learned draft's are the first phase's neighbours within its largest cutoff (no lanes idle on
            // candidates outside it during the radial adjoint)
            const int *nrow = w_nbr + (size_t)i * ccap;
            const int nc2 = LEARNED ? __ldcg(w_nbr + (size_t)N * ccap + i) : nl;
            for (int t0 = lane; t0 < ((!LEARNED && minimg) ? 0 : nc2); t0 += 128) {
                int kq[4];
                uint4 fq[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int t = t0 + 32 * u;
                    kq[u] = t < nc2 ? (LEARNED ? __ldcg(nrow + t) : (use_list ? lst[t] : t)) : i;
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) fq[u] = kq[u] != i ? fx[kq[u]] : fi;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (t0 + 32 * u >= nc2) break;
                    const int k = kq[u];
                    if (k == i) continue;
                    const uint4 fk = fq[u];
                    const int pr2 = si * g.S + (int)fk.w;
                    const float sig2 = slj[pr2], eps24 = slj[kMaxSpecies * kMaxSpecies + pr2];
                    for_images(g, fi, fk, rc2_all, minimg != 0, [&](float dx, float dy, float dz, float d2) {
                        // the learned draft: 1/r once per pair (its cutoff spans the LJ one)
                        const float ir = LEARNED ? rsqrtf(d2) : 0.f;
                        if (P.has_lj && d2 < P.lj_rc2f) {
                            const float inv = LEARNED ? ir * ir : 1.f / d2;
                            const float s2 = sig2 * inv;
                            const float s6 = s2 * s2 * s2, s12 = s6 * s6;
                            const float fr = -eps24 * (2.f * s12 - s6) * inv;
                            fxx += fr * dx;
                            fyy += fr * dy;
                            fzz += fr * dz;
                        }
                        if (LEARNED && d2 < P.desc_rc2f) {
                            // radial adjoint in gather form: (c_ik + c_ki) d/r
                            const float r = d2 * ir;
                            float fc, dfc;
                            draft_cutoff(r, inv_rc, fc, dfc);
                            float cc = 0.f;
                            if (stage_dedx) {
                                const int SR = g.S * P.n_rbf;
                                const float *gi = sdedx + (size_t)i * SR + (int)fk.w * P.n_rbf;
                                const float *gk = sdedx + (size_t)k * SR + si * P.n_rbf;
                                for (int b = 0; b < P.n_rbf; ++b) {
                                    const float tt = r - (float)b * P.rbf_w;
                                    const float dg = __expf(-tt * tt * P.rbf_inv2w2) * (-tt * P.rbf_invw2 * fc + dfc);
                                    cc += (gi[b] + gk[b]) * dg;
                                }
                            } else if ((P.n_rbf & 3) == 0 && (P.d0p & 3) == 0) {
                                // both atoms' blocks of dE/dX through L2, four basis functions per 16-byte load
                                const float4 *gi = reinterpret_cast<const float4 *>(w_dEdX + (size_t)i * P.d0p +
                                                                                    (int)fk.w * P.n_rbf);
                                const float4 *gk = reinterpret_cast<const float4 *>(w_dEdX + (size_t)k * P.d0p +
                                                                                    si * P.n_rbf);
                                auto block4 = [&](int b4) {
                                    const float4 a = __ldcg(gi + b4), c = __ldcg(gk + b4);
                                    const float gs[4] = {a.x + c.x, a.y + c.y, a.z + c.z, a.w + c.w};
#pragma unroll
                                    for (int e = 0; e < 4; ++e) {
                                        const float tt = r - (float)(4 * b4 + e) * P.rbf_w;
                                        const float dg = __expf(-tt * tt * P.rbf_inv2w2) * (-tt * P.rbf_invw2 * fc + dfc);
                                        cc += gs[e] * dg;
                                    }
                                };
                                if (P.n_rbf == 8) {   // the usual basis: both blocks' loads issued together
                                    block4(0);
                                    block4(1);
                                } else {
                                    for (int b4 = 0; b4 < P.n_rbf / 4; ++b4) block4(b4);
                                }
                            } else {
                                const float *gi = w_dEdX + (size_t)i * P.d0p + (int)fk.w * P.n_rbf;
                                const float *gk = w_dEdX + (size_t)k * P.d0p + si * P.n_rbf;
                                for (int b = 0; b < P.n_rbf; ++b) {
                                    const float tt = r - (float)b * P.rbf_w;
                                    const float dg = __expf(-tt * tt * P.rbf_inv2w2) * (-tt * P.rbf_invw2 * fc + dfc);
                                    cc += (__ldcg(gi + b) + __ldcg(gk + b)) * dg;
                                }
                            }
                            const float cr = cc * ir;
                            fxx += cr * dx;
                            fyy += cr * dy;
                            fzz += cr * dz;
                        }
                    });
                }
            }
            // the three warp sums in six shuffles: halves exchange pairs of
            // components, quarters single ones, then an ordinary butterfly;
            // lanes 0, 8 and 16 end with the x, y and z totals
            {
                const bool lo = lane < 16;
                float k0 = lo ? fxx : fzz, k1 = lo ? fyy : 0.f;
                const float s0 = lo ? fzz : fxx, s1 = lo ? 0.f : fyy;
                k0 += __shfl_xor_sync(0xffffffffu, s0, 16);
                k1 += __shfl_xor_sync(0xffffffffu, s1, 16);
                const bool q = (lane & 8) != 0;
                float v = q ? k1 : k0;
                v += __shfl_xor_sync(0xffffffffu, q ? k0 : k1, 8);
                v += __shfl_xor_sync(0xffffffffu, v, 4);
                v += __shfl_xor_sync(0xffffffffu, v, 2);
                v += __shfl_xor_sync(0xffffffffu, v, 1);
                if ((lane & 7) == 0 && lane < 24) (&sF[ii].x)[lane >> 3] = v;
            }
        }
        __syncthreads();
        // the flag of this parity is next written (by any CTA) after the next barrier
        if (!GRID && use_list && !stage_fix && tid == 0) sflag[par] = 0;
        // D: BOB + A, one lane per coordinate
        auto step_d = [&](int p, double &preg, float dfreg, float xreg, double c1p_r, double sxi_r) {
            const int ii = grp + p * kGroups;
            if (ii >= nown || x >= 3) return;
            const int i = a0 + ii;
            const int sp = sspec[ii];
            const float4 F = sF[ii];
            const float fr = x == 0 ? F.x : (x == 1 ? F.y : F.z);
            float xx = xreg;
            if (noise_smem) {
                xx = snoise[((size_t)jl * A + ii) * 3 + x];
            } else if (!REG) {
                const float3 xi = normals3(cf.seed, n, (uint32_t)i, 0u);
                xx = x == 0 ? xi.x : (x == 1 ? xi.y : xi.z);
            }
            const size_t o = (size_t)j * D + 3 * i + x;
            const double pv = REG ? preg : ((j == 0) ? p_base[3 * i + x] : w_pdraft[o - D]);
            const float fu = ec_on ? fr + (REG ? dfreg : ec_dF[3 * i + x]) : fr;
            const double mu = __dadd_rn(REG ? c1p_r : __dmul_rn(cf.c1, pv), __dmul_rn(cf.aF, (double)fu));
            const double pn = __dadd_rn(mu, REG ? sxi_r : __dmul_rn(species_pick(cf.sig, sp), (double)xx));
            if (REG) preg = pn;
            w_pdraft[o] = pn;
            w_Fd[o] = fu;
            if (ec_on) w_Fraw[o] = fr;
        };
        if (REG) {
#pragma unroll
            for (int p = 0; p < kP; ++p)
                if (p < passes) step_d(p, pr[p], dfr[p], xr[p], c1p[p], sxi[p]);
        } else {
            double dp;
            for (int p = 0; p < passes; ++p) step_d(p, dp, 0.f, 0.f, 0.0, 0.0);
        }
        // the next step reads owned atoms' state from this thread's registers or
        // its own global writes, and sF is rewritten only after the next cluster
        // barrier: no CTA barrier is needed here
    }
    if (gave_up) {
        // A CTA that gave up may still be the target of its peers' stores of the
        // next step (they received this step's positions and went on).  Those
        // peers then give up on that step themselves, two seconds later, and
        // come here too: each CTA that gave up arrives on every CTA's exit
        // barrier and waits, three times as long, for all C arrivals before it
        // exits, so no peer that is still sending finds it gone.  Peers that
        // stopped normally at this step send nothing more; the wait then runs
        // out and the CTA exits (the window already carries the error bit).
        if (tid < C)
            asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(
                             tc::cluster_map(bar0 + 16, (uint32_t)tid))
                         : "memory");
        if (tid == 0) {
            const long long t0 = clock64();
            while (!tc::mbar_try_wait_cluster(bar0 + 16, 0u) && clock64() - t0 < 12000000000ll) {
            }
        }
        __syncthreads();
    }
    if (c == 0 && tid == 0) {
        if (hdr) {
            hdr->k_eff = keff;
            if (redraft) {
                hdr->base = n0;
                hdr->skip = 0;
            }
        } else {
            st->k_eff = keff;
        }
    }
}

static size_t draft_smem_bytes(int N, int C, const PotDev &P, bool learned, bool stage_fix, int noise_K, int vcap,
                               bool stage_list, size_t dedx_floats) {
    // vcap > 0: lists (global or built in the kernel), each CTA's list bases staged
    const int A = (N + C - 1) / C;
    size_t b = (size_t)A * sizeof(float4) + 2 * kMaxSpecies * kMaxSpecies * sizeof(float);
    if (vcap > 0) b += (size_t)A * sizeof(uint4);
    b += (size_t)A * sizeof(int);
    if (stage_list) b += (size_t)A * (vcap + 1) * sizeof(int);
    if (learned) {
        const int S = P.n_rbf > 0 ? (P.d0 - P.n_ang) / (P.n_rbf + 1) : 0;   // input = S n_rbf radial + one-hot S
        b += ((size_t)kDraftWarps * learned_stage_floats(S, P.d0p) + learned_weight_floats(P.d0p)) * sizeof(float);
    }
    if (stage_fix) b += 2 * (size_t)N * sizeof(uint4);
    return b + 2 * kMaxCluster * sizeof(int) + 3 * sizeof(uint64_t) + (size_t)noise_K * A * 3 * sizeof(float) +
           dedx_floats * sizeof(float);
}

constexpr size_t kNoiseSmemMax = 32 * 1024;   // the window's noise is staged up front when it fits
constexpr size_t kListSmemMax = 64 * 1024;    // owned atoms' Verlet lists are staged when they fit
constexpr size_t kDedxSmemMax = 48 * 1024;    // the learned draft's radial dE/dX of all atoms, staged when it fits

DraftPlan draft_plan(int N, int K, const PotDev &P, bool learned, int vcap, bool all_pairs, int max_cluster,
                     size_t max_smem) {
    DraftPlan pl{};
    int C = 1;
    max_cluster = max_cluster < kMaxCluster ? max_cluster : kMaxCluster;
    while (C < max_cluster && (N + C - 1) / C > 16) C *= 2;
    pl.cluster = C;
    pl.stage_fix = 2 * (size_t)N * sizeof(uint4) <= 128 * 1024;
    pl.noise_step_bytes = (size_t)((N + C - 1) / C) * 3 * sizeof(float);
    pl.K = K;
    pl.stage_list = vcap > 0 && (size_t)((N + C - 1) / C) * (vcap + 1) * sizeof(int) <= kListSmemMax;
    // without a cell grid the kernel lists candidates itself when the lists fit
    // (and the base positions fit in the staged position buffers)
    pl.self_list = all_pairs && pl.stage_list && pl.stage_fix;
    if (all_pairs && !pl.self_list) {
        vcap = 0;   // every atom is a candidate; no lists at all
        pl.stage_list = false;
    }
    // the learned draft's radial dE/dX of every atom, staged per step when it is small
    const int S = P.n_rbf > 0 ? (P.d0 - P.n_ang) / (P.n_rbf + 1) : 0;
    const size_t dedx = (size_t)N * S * P.n_rbf;
    pl.stage_dedx = learned && dedx > 0 && dedx * sizeof(float) <= kDedxSmemMax;
    pl.smem_base = draft_smem_bytes(N, C, P, learned, pl.stage_fix, 0, vcap, pl.stage_list, pl.stage_dedx ? dedx : 0);
    pl.max_smem = max_smem;
    draft_plan_noise(pl, K);
    pl.reg = (N + C - 1) / C <= kRegPasses * kGroups;
    pl.ok = pl.smem <= max_smem;
    return pl;
}

// The grid form: one CTA per SM, positions through L2, the window's Verlet
// lists (a cell grid is required: without one every atom would be every
// CTA's candidate).
DraftPlan draft_grid_plan(int N, int K, const PotDev &P, bool learned, int vcap, bool all_pairs, int n_sm,
                          size_t max_smem) {
    DraftPlan pl{};
    if (all_pairs || vcap <= 0 || n_sm <= 0) return pl;
    const int C = n_sm < N ? n_sm : N;
    const int A = (N + C - 1) / C;
    pl.cluster = C;
    pl.grid = true;
    pl.stage_fix = false;
    pl.self_list = false;
    pl.K = K;
    pl.noise_step_bytes = (size_t)A * 3 * sizeof(float);
    pl.stage_list = (size_t)A * (vcap + 1) * sizeof(int) <= kListSmemMax;
    const int S = P.n_rbf > 0 ? (P.d0 - P.n_ang) / (P.n_rbf + 1) : 0;
    const size_t dedx = (size_t)N * S * P.n_rbf;
    pl.stage_dedx = learned && dedx > 0 && dedx * sizeof(float) <= kDedxSmemMax;
    pl.smem_base = draft_smem_bytes(N, C, P, learned, false, 0, vcap, pl.stage_list, pl.stage_dedx ? dedx : 0);
    pl.max_smem = max_smem;
    draft_plan_noise(pl, K);
    pl.reg = A <= kRegPasses * kGroups;
    return pl;
}

void draft_plan_noise(DraftPlan &pl, int steps) {
    pl.noise_steps = (size_t)steps * pl.noise_step_bytes <= kNoiseSmemMax ? steps : 0;
    pl.smem = pl.smem_base + (size_t)pl.noise_steps * pl.noise_step_bytes;
    pl.ok = pl.smem <= pl.max_smem;
}

cudaError_t launch_draft(const DraftPlan &pl, bool learned, int K, const Geo &g, const PotDev &P, const Coef &cf,
                         const VerletPlan &vp, const VerletBufs &vb, const int *species, const double *q,
                         const double *p, const float *ec_dF, int ec_on, DevState *st, double *w_qmid,
                         double *w_pdraft, float *w_Fd, float *w_Fraw, uint4 *w_fix, float *w_dEdX,
                         cudaStream_t s, WinHdr *hdr, int redraft, DraftSync *sync, int j0, int *w_nbr, int ccap) {
    if (learned && (!w_nbr || ccap <= 0)) return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(pl.cluster, 1, 1);
    cfg.blockDim = dim3(kDraftThreads, 1, 1);
    cfg.dynamicSmemBytes = pl.smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    if (pl.grid) {
        if (!sync) return cudaErrorInvalidValue;
        const cudaError_t e = cudaMemsetAsync(sync, 0, sizeof(DraftSync), s);
        if (e != cudaSuccess) return e;
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
    } else {
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = pl.cluster;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
    }
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const int stage = pl.stage_fix ? 1 : 0;
    const int *vl = vp.all_pairs ? nullptr : (const int *)vb.vlist;
    const int mi = pl.minimg ? 1 : 0;
    const int ns = (K - j0 <= pl.noise_steps) ? 1 : 0;   // this launch drafts steps j0 .. K - 1
    const int self = (pl.self_list && vp.all_pairs) ? 1 : 0;
    const int sl = (pl.stage_list && (vl || self)) ? 1 : 0;
    const int sd = (learned && pl.stage_dedx) ? 1 : 0;
    using Kern = decltype(&draft_window_cluster_kernel<false, false, false>);
    static const Kern kerns[8] = {
        draft_window_cluster_kernel<false, false, false>, draft_window_cluster_kernel<false, true, false>,
        draft_window_cluster_kernel<true, false, false>,  draft_window_cluster_kernel<true, true, false>,
        draft_window_cluster_kernel<false, false, true>,  draft_window_cluster_kernel<false, true, true>,
        draft_window_cluster_kernel<true, false, true>,   draft_window_cluster_kernel<true, true, true>};
    const Kern kern = kerns[(pl.grid ? 4 : 0) + (learned ? 2 : 0) + (pl.reg ? 1 : 0)];
    return cudaLaunchKernelEx(&cfg, kern, K, g, P, cf, vl, (const int *)vb.vcount, vp.cap, (const uint4 *)vb.fix_base,
                              vp.move2f, vp.rlist2f, stage, mi, ns, sl, self, sd, species, q, p, ec_dF, ec_on, st, w_qmid, w_pdraft, w_Fd,
                              w_Fraw, w_fix, w_dEdX, w_nbr, ccap, hdr, redraft, sync, j0);
}

static const void *draft_kernel_ptrs[8] = {
    (const void *)draft_window_cluster_kernel<false, false, false>,
    (const void *)draft_window_cluster_kernel<false, true, false>,
    (const void *)draft_window_cluster_kernel<true, false, false>,
    (const void *)draft_window_cluster_kernel<true, true, false>,
    (const void *)draft_window_cluster_kernel<false, false, true>,
    (const void *)draft_window_cluster_kernel<false, true, true>,
    (const void *)draft_window_cluster_kernel<true, false, true>,
    (const void *)draft_window_cluster_kernel<true, true, true>};

cudaError_t draft_kernels_setup(int max_smem) {
    for (const void *k : draft_kernel_ptrs) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Every CTA of the grid form resident at once (the cooperative launch's condition).
bool draft_grid_fits(const DraftPlan &pl, bool learned, int n_sm) {
    int per_sm = 0;
    const void *k = draft_kernel_ptrs[4 + (learned ? 2 : 0) + (pl.reg ? 1 : 0)];
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kDraftThreads, pl.smem) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return per_sm * n_sm >= pl.cluster;
}

int draft_max_cluster(size_t smem, bool learned) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(16, 1, 1);
    cfg.blockDim = dim3(kDraftThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 16;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int c = 0;
    const void *k = draft_kernel_ptrs[learned ? 3 : 1];
    if (cudaOccupancyMaxPotentialClusterSize(&c, k, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 8;
    }
    return c >= 16 ? 16 : (c >= 8 ? 8 : (c >= 4 ? 4 : (c >= 2 ? 2 : 1)));
}

// ---------------------------------------------------------------------------
// The pipelined window loop (single-GPU form of the pipelined protocol of
// Alg. 2): while window b is verified, window b^1 is drafted speculatively
// from the last drafted state of b, as if all of b were accepted.  After the
// verification the speculative draft is kept iff its base step equals the
// committed step and b had no rejection (then every step of b was accepted and
// the committed state is the speculative base bit for bit, so the draft is the
// one a fresh start would make); otherwise b^1 is drafted again from the
// committed state.
// ---------------------------------------------------------------------------

// The speculative base of window b^1: the state after the last step window b
// drafted (ABOBA: q_mid + (dt/2) p/m with the commit's rounding; staggered
// OBABO: q_mid), its step index, and whether there is one (k_eff > 0).  The
// speculative draft is skipped (it would not stand: every recent window had a
// rejection) when the policy of the previous round says so (st->spec_hint,
// written by this stream's redraft test after the previous commit).
__global__ void spec_base_kernel(Geo g, Coef cf, const int *__restrict__ species, const double *__restrict__ qmid_b,
                                 const double *__restrict__ pdraft_b, const WinHdr *__restrict__ hb,
                                 WinHdr *__restrict__ hn, const DevState *__restrict__ st, double *__restrict__ qb,
                                 double *__restrict__ pb) {
    const int k = hb->k_eff;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) {
        hn->base = k > 0 ? hb->base + k : -1;
        hn->skip = (k > 0 && st->spec_hint == 0) ? 0 : 1;
    }
    if (k <= 0 || i >= g.N) return;
    const size_t o = (size_t)(k - 1) * 3 * g.N + 3 * (size_t)i;
    const double hm = species_pick(cf.hm, species[i]);
#pragma unroll
    for (int x = 0; x < 3; ++x) {
        const double pn = pdraft_b[o + x];
        pb[3 * i + x] = pn;
        qb[3 * i + x] = cf.obabo ? qmid_b[o + x] : __dadd_rn(qmid_b[o + x], __dmul_rn(pn, hm));
    }
}


// The redraft's Verlet build runs only when the speculative draft does not
// stand (the same test the redraft itself makes).  Then the speculation
// policy of the next round: a speculative draft stands only after a window
// with no rejection, so the next round drafts speculatively while the running
// mean of that event (weight 1/4 for the window just committed) is at least
// 0.2.  The policy changes only which work runs, never the result: a skipped
// speculation is a redraft from the committed state, the unpipelined loop's
// draft.  Only kernels of the draft stream read or write spec_ema and
// spec_hint.
__global__ void redraft_flag_kernel(DevState *__restrict__ st, WinHdr *__restrict__ hn) {
    hn->keep = spec_is_valid(hn, st) ? 1 : 0;
    const float e = 0.75f * st->spec_ema + (st->first_reject_last == -1 ? 0.25f : 0.f);
    st->spec_ema = e;
    st->spec_hint = e < 0.2f ? 1 : 0;
}

__global__ void hdr_invalidate_kernel(WinHdr *__restrict__ h) {
    h->base = -1;
    h->skip = 1;
    h->k_eff = 0;
}

void launch_spec_base(const Geo &g, const Coef &cf, const int *species, const double *qmid_b, const double *pdraft_b,
                      const WinHdr *hb, WinHdr *hn, const DevState *st, double *qb, double *pb, cudaStream_t s) {
    spec_base_kernel<<<(g.N + 255) / 256, 256, 0, s>>>(g, cf, species, qmid_b, pdraft_b, hb, hn, st, qb, pb);
}

void launch_redraft_flag(DevState *st, WinHdr *hn, cudaStream_t s) { redraft_flag_kernel<<<1, 1, 0, s>>>(st, hn); }


void launch_hdr_invalidate(WinHdr *h, cudaStream_t s) { hdr_invalidate_kernel<<<1, 1, 0, s>>>(h); }

// ---------------------------------------------------------------------------
// Plain target ABOBA (the baseline): half step before the batched force
// evaluation, BOB + A after it.  Multi-CTA; the last CTA advances the step.
// ---------------------------------------------------------------------------
__global__ void plain_half_kernel(Geo g, Coef cf, const int *__restrict__ species, const double *__restrict__ q,
                                  const double *__restrict__ p, DevState *__restrict__ st,
                                  double *__restrict__ qmid, uint4 *__restrict__ fix) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (st->step >= st->target_step || i >= g.N) return;
    if (i == 0) st->k_eff = 1;   // one step, always inside the lists' skin
    const int sp = species[i];
    const double hm = cf.obabo ? species_pick(cf.hmf, sp) : species_pick(cf.hm, sp);
    uint32_t u0, u1, u2;
#pragma unroll
    for (int x = 0; x < 3; ++x) {
        const double qm = __dadd_rn(q[3 * i + x], __dmul_rn(p[3 * i + x], hm));
        qmid[3 * i + x] = qm;
        const uint32_t u = fixpoint(qm, g.scale[x]);
        if (x == 0) u0 = u; else if (x == 1) u1 = u; else u2 = u;
    }
    fix[i] = make_uint4(u0, u1, u2, (unsigned)sp);
}

__global__ void plain_finish_kernel(Geo g, Coef cf, const int *__restrict__ species, const double *__restrict__ qmid,
                                    const float *__restrict__ F, double *__restrict__ q, double *__restrict__ p,
                                    double *__restrict__ p_obabo, DevState *__restrict__ st) {
    __shared__ bool s_last;
    if (st->step >= st->target_step) return;
    const long long n0 = st->step;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < g.N) {
        const int sp = species[i];
        const float3 xi = normals3(cf.seed, (unsigned long long)(n0 + 1), (uint32_t)i, 0u);
#pragma unroll
        for (int x = 0; x < 3; ++x) {
            const int o = 3 * i + x;
            const float xx = x == 0 ? xi.x : (x == 1 ? xi.y : xi.z);
            const double pprev = p[o];
            const double mu = __dadd_rn(__dmul_rn(cf.c1, pprev), __dmul_rn(cf.aF, (double)F[o]));
            const double pn = __dadd_rn(mu, __dmul_rn(species_pick(cf.sig, sp), (double)xx));
            p[o] = pn;
            if (cf.obabo) {
                q[o] = qmid[o];
                const float3 eta = normals3(cf.seed, (unsigned long long)(n0 + 1), (uint32_t)i, 3u);
                p_obabo[o] = obabo_output(cf, sp, pprev, (double)F[o], pn, x == 0 ? eta.x : (x == 1 ? eta.y : eta.z));
            } else {
                q[o] = __dadd_rn(qmid[o], __dmul_rn(pn, species_pick(cf.hm, sp)));
            }
        }
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(&st->blocks_done, 1u) == gridDim.x - 1);
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
        __threadfence();
        st->blocks_done = 0u;
        st->step = n0 + 1;
    }
}

void launch_plain_half(const Geo &g, const Coef &cf, const int *species, const double *q, const double *p,
                       DevState *st, double *qmid, uint4 *fix, cudaStream_t s) {
    plain_half_kernel<<<(g.N + 255) / 256, 256, 0, s>>>(g, cf, species, q, p, st, qmid, fix);
}

void launch_plain_finish(const Geo &g, const Coef &cf, const int *species, const double *qmid, const float *F,
                         double *q, double *p, double *p_obabo, DevState *st, cudaStream_t s) {
    plain_finish_kernel<<<(g.N + 255) / 256, 256, 0, s>>>(g, cf, species, qmid, F, q, p, p_obabo, st);
}

// Enters the staggered OBABO frame from an OBABO state at step index n: the
// leading O half-step (noise stream 4 at n) and B half-step with the target
// force F at q, p <- (e^(-gamma dt/2) p + Sigma_1/2^1/2 xi) + (dt/2) kappa F.
__global__ void obabo_enter_kernel(Geo g, Coef cf, const int *__restrict__ species, const float *__restrict__ F,
                                   long long n, double *__restrict__ p) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.N) return;
    const int sp = species[i];
    const float3 xi = normals3(cf.seed, (unsigned long long)n, (uint32_t)i, 4u);
    const double sh = species_pick(cf.sigh, sp);
#pragma unroll
    for (int x = 0; x < 3; ++x) {
        const int o = 3 * i + x;
        const double xx = x == 0 ? xi.x : (x == 1 ? xi.y : xi.z);
        p[o] = __dadd_rn(__dadd_rn(__dmul_rn(cf.ch, p[o]), __dmul_rn(sh, xx)), __dmul_rn(cf.bF, (double)F[o]));
    }
}

void launch_obabo_enter(const Geo &g, const Coef &cf, const int *species, const float *F, long long n, double *p,
                        cudaStream_t s) {
    obabo_enter_kernel<<<(g.N + 255) / 256, 256, 0, s>>>(g, cf, species, F, n, p);
}

}  // namespace lsd
