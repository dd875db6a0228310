// lsd_transport.cu -- reflectionVerify (Eq. 5) on every window step, the first
// rejection (Alg. 1), and the rollback/commit of the state.
//
// With z = S^-1/2 (p~ - <p~>) = xi (the draft's own noise, regenerated from
// its counter) and delta = S^-1/2 (<p~> - <p>) = (1+c1)(dt/2) kappa (F~ - F)/sigma
// (the c1 p terms of both means cancel), the log density ratio is
// log r = -z.delta - |delta|^2/2; a step is accepted iff log u <= min(0, log r).
// A rejected step's momentum is <p> + sigma (z - 2 (z.delta/delta.delta) delta)
// and its position q_mid + (dt/2) p/m (the shared map g = A of Thm 3.1).
//
// transport_reduce_kernel: per (chunk of atoms, window step) partial sums of
//   z.delta and delta.delta, written to a fixed slot (no atomics).  Everything
//   from the first product up is FP64: delta's components are FP64 products of
//   the exact FP64 difference of the two FP32 forces, z is the FP32 normal
//   widened exactly, and the sums over an atom's three components, a warp's
//   32 atoms, the warps, the chunks and the log ratio are FP64 in a fixed
//   order.  log u (one FP64 log per step) is formed by the deciding kernel
//   itself; the cooperative form does it before its wait on the force
//   gather, so it overlaps the gather.
// transport_commit_kernel: every CTA sums the partials in the same fixed
//   order, finds l = first rejected step, and commits its slice of atoms:
//   the draft's own bits for an accepted step, the reflection for a rejected
//   one.  The last CTA to finish advances the step counter and statistics.
#include "lsd_common.cuh"
#include "lsd_kernels.h"

namespace lsd {

constexpr int kTransThreads = 256;

// The block's FP64 sums of a and b in a fixed order: a butterfly within each
// warp, then warp 0 over the warps' results.
__device__ __forceinline__ double2 block_sum2(double a, double b, double2 *sh) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    a = warp_sum_d(a);
    b = warp_sum_d(b);
    if (lane == 0) sh[w] = make_double2(a, b);
    __syncthreads();
    double2 t = make_double2(0.0, 0.0);
    if (w == 0) {
        if (lane < nw) t = sh[lane];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            t.x += __shfl_down_sync(0xffffffffu, t.x, o);
            t.y += __shfl_down_sync(0xffffffffu, t.y, o);
        }
    }
    return t;   // valid in thread 0
}

// One atom's terms of z.delta and delta.delta, added to s and d, all in FP64:
// delta_c = k (F~_c - F_c) with k = (1+c1)(dt/2) kappa / sigma of its species
// (the FP64 difference of two FP32 values is exact), z_c = xi_c.
__device__ __forceinline__ void atom_terms(double k, float3 xi, float3 fd, const float *__restrict__ ft, double &s,
                                           double &d) {
    const double d0 = k * ((double)fd.x - (double)ft[0]);
    const double d1 = k * ((double)fd.y - (double)ft[1]);
    const double d2 = k * ((double)fd.z - (double)ft[2]);
    s += ((double)xi.x * d0 + (double)xi.y * d1) + (double)xi.z * d2;
    d += (d0 * d0 + d1 * d1) + d2 * d2;
}

// Shared state of a window's decision, used by the commit (and by the fused
// reduce-commit for windows whose atoms fit in one block).
struct CommitShared {
    double s[kMaxK], d[kMaxK], lr[kMaxK], lu[kMaxK], dn[kMaxK], pr[kMaxK];
    int acc[kMaxK], fin[kMaxK];
    int nc, rej, l, bad;
    double factor;   // 2 z.delta / delta.delta of the committed step when it was rejected
};

// log u of the acceptance test of window steps 0..K-1 (one FP64 log each),
// into C.lu, by thread j % blockDim.x -- the thread that reads it in
// commit_decide, so no barrier is needed in between.
__device__ __forceinline__ void logu_fill(CommitShared &C, const Coef &cf, long long n0, int K) {
    for (int j = threadIdx.x; j < K; j += blockDim.x) C.lu[j] = log(uniform53(cf.seed, (unsigned long long)(n0 + j + 1)));
}

// Sums the partials of every window step in a fixed order, forms log r and
// the accept flags (against C.lu, filled by logu_fill), and finds l = the
// first rejected step (all threads).
__device__ void commit_decide(CommitShared &C, int K, const double2 *__restrict__ partials, int n_part,
                              long long rem) {
    for (int j = threadIdx.x; j < K; j += blockDim.x) {
        double s = 0.0, d = 0.0;
        for (int b = 0; b < n_part; ++b) {
            const double2 v = __ldcg(partials + (size_t)j * n_part + b);
            s += v.x;
            d += v.y;
        }
        C.s[j] = s;
        C.d[j] = d;
        const double lr = -s - 0.5 * d;
        const double lu = C.lu[j];
        C.lr[j] = lr;
        C.acc[j] = (d == 0.0) || (lu <= fmin(0.0, lr));
        C.fin[j] = isfinite(lr);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int l = K, rej = 0, bad = 0;
        for (int j = 0; j < K; ++j) {
            if (!C.fin[j]) { bad = 1; l = j + 1; break; }
            if (!C.acc[j]) { l = j + 1; rej = 1; break; }
        }
        const int nc = (long long)l < rem ? l : (int)rem;
        C.l = l;
        C.nc = bad ? 0 : nc;
        C.rej = (rej && nc == l) ? 1 : 0;
        C.bad = bad;
        C.factor = C.rej ? 2.0 * C.s[nc - 1] / C.d[nc - 1] : 0.0;
    }
    __syncthreads();
}

// A window verified in stages (lsd_set_window_stages): after stage s the
// window goes on to stage s + 1 (a conditional graph node, `next`) only when
// every step so far was accepted, the draft reached the stage's end and the
// stop step lies beyond it; then nothing is committed yet.  Otherwise the
// window ends here with the commit an unstaged window would make: the first
// rejection decides, and the steps past it are never verified.
__device__ __forceinline__ bool stage_continues(const CommitShared &C, int Kw, int K, int staged, long long rem) {
    return staged && !C.bad && !C.rej && Kw == K && (long long)Kw < rem;
}
__device__ __forceinline__ void stage_signal(cudaGraphConditionalHandle next) { cudaGraphSetConditional(next, 1u); }

// Commits atoms [a0, a1): the draft's own bits for an accepted last step, the
// reflection (Eq. 5) for a rejected one; the staggered OBABO frame keeps the
// position and recovers the output momentum (App. E).
__device__ void commit_atoms(const CommitShared &C, int N, const Coef &cf, const int *__restrict__ species,
                             const double *__restrict__ w_qmid, const double *__restrict__ w_pdraft,
                             const float *__restrict__ Fd, const float *__restrict__ Ft,
                             const float *__restrict__ Fraw, float *__restrict__ ec_dF, int ec_on,
                             double *__restrict__ q, double *__restrict__ p, double *__restrict__ p_obabo,
                             long long n0, int a0, int a1) {
    const int nc = C.nc;
    if (nc <= 0) return;
    const int jj = nc - 1;
    const size_t D = (size_t)3 * N;
    const double factor = C.factor;
    const unsigned long long n = (unsigned long long)(n0 + jj + 1);
    for (int i = a0 + threadIdx.x; i < a1; i += blockDim.x) {
        const int sp = species[i];
        const double hm = species_pick(cf.hm, sp);
        float3 xi = make_float3(0.f, 0.f, 0.f);
        if (C.rej) xi = normals3(cf.seed, n, (uint32_t)i, 0u);
        float3 eta = make_float3(0.f, 0.f, 0.f);
        if (cf.obabo) eta = normals3(cf.seed, n, (uint32_t)i, 3u);
        const float xs[3] = {xi.x, xi.y, xi.z}, es[3] = {eta.x, eta.y, eta.z};
        for (int c = 0; c < 3; ++c) {
            const size_t o = (size_t)jj * D + (size_t)3 * i + c;
            const double pprev = jj == 0 ? p[3 * i + c] : w_pdraft[o - D];
            double pn;
            if (C.rej) {
                const double mu = __dadd_rn(__dmul_rn(cf.c1, pprev), __dmul_rn(cf.aF, (double)Ft[o]));
                const double dl = species_pick(cf.aF_sig, sp) * ((double)Fd[o] - (double)Ft[o]);
                pn = mu + species_pick(cf.sig, sp) * ((double)xs[c] - factor * dl);
            } else {
                pn = w_pdraft[o];
            }
            p[3 * i + c] = pn;
            if (cf.obabo) {
                // staggered frame: no trailing A; the OBABO output of the committed step (App. E)
                q[3 * i + c] = w_qmid[o];
                p_obabo[3 * i + c] = obabo_output(cf, sp, pprev, (double)Ft[o], pn, (double)es[c]);
            } else {
                q[3 * i + c] = __dadd_rn(w_qmid[o], __dmul_rn(pn, hm));
            }
            if (ec_on) ec_dF[3 * i + c] = Ft[o] - Fraw[o];
        }
    }
}

// Statistics of the window and the step advance (one block, all threads).
// K: the window's drafted steps (k_eff, at most Kl, the steps the launch
// covers).  A window that committed every drafted step, none reflected, and
// was drafted short of Kl ended at the draft's displacement bound: kept lists
// (lsd_set_list_reuse) are rebuilt before the next window.
__device__ void commit_stats(CommitShared &C, int K, DevState *__restrict__ st, long long n0, int Kl) {
    const int nc = C.nc;
    for (int j = threadIdx.x; j < K; j += blockDim.x) {
        const double dn = sqrt(C.d[j]);
        C.dn[j] = dn;
        C.pr[j] = (double)erff((float)dn * 0.35355339059327373f);   // erf(|delta| / sqrt 8), Eq. 6
        st->accept[j] = C.acc[j];
        st->logr[j] = C.lr[j];
        st->logu[j] = C.lu[j];
        st->dnorm[j] = dn;
    }
    __syncthreads();
    double sd = 0.0, sp = 0.0;
    if (threadIdx.x < 32) {
        for (int j = threadIdx.x; j < nc; j += 32) {
            sd += C.dn[j];
            sp += C.pr[j];
        }
        sd = warp_sum_d(sd);
        sp = warp_sum_d(sp);
    }
    if (threadIdx.x == 0) {
        st->n_commit_last = nc;
        st->k_eff = K;   // the window's drafted steps (a pipelined round reads them from its header)
        st->first_reject_last = C.rej || (C.l <= K && !C.acc[C.l - 1]) ? C.l : -1;
        if (C.bad) atomicOr(&st->err, 2);
        st->windows += 1;
        st->verified += K;
        st->stages += 1;
        if (nc == K && !C.rej && K < Kl) st->list_force = 1;
        st->committed += nc;
        st->rejected += C.rej;
        st->sum_delta += sd;
        st->sum_pred += sp;
        st->step = n0 + nc;
    }
}

// Per window step j (blockIdx.y) and slice of atoms (blockIdx.x): z.delta and
// delta.delta, with delta = (1+c1)(dt/2)kappa (F~ - F) / sigma and z = xi (the
// draft's own noise).  fused:
// the window's atoms fit in one block, and the last block to finish decides,
// commits every atom and updates the statistics (no second launch).
__global__ void __launch_bounds__(kTransThreads)
    transport_reduce_kernel(int K, Geo g, Coef cf, const int *__restrict__ species, const float *__restrict__ Fd,
                            const float *__restrict__ Ft, DevState *__restrict__ st, double2 *__restrict__ partials,
                            const int *__restrict__ keff_p, int atoms_per_block, int fused,
                            const double *__restrict__ w_qmid, const double *__restrict__ w_pdraft,
                            const float *__restrict__ Fraw, float *__restrict__ ec_dF, int ec_on,
                            double *__restrict__ q, double *__restrict__ p, double *__restrict__ p_obabo, int j0,
                            int staged, cudaGraphConditionalHandle next) {
    __shared__ double2 sh[32];
    __shared__ CommitShared C;
    __shared__ bool s_last;
    pdl_wait();
    pdl_release();
    if (st->step >= st->target_step) return;   // uniform over the grid
    const int N = g.N;
    const int j = j0 + blockIdx.y;             // window steps j0 .. K - 1 (earlier stages reduced the others)
    const int keff = *keff_p;
    if (j < keff) {                            // steps the draft did not reach are skipped
        const unsigned long long n = (unsigned long long)(st->step + j + 1);
        const int a0 = blockIdx.x * atoms_per_block;
        const int a1 = min(N, a0 + atoms_per_block);
        double s = 0.0, d = 0.0;
        for (int i = a0 + threadIdx.x; i < a1; i += blockDim.x) {
            const float3 xi = normals3(cf.seed, n, (uint32_t)i, 0u);
            const double k = species_pick(cf.aF_sig, species[i]);
            const size_t o = ((size_t)j * N + i) * 3;
            atom_terms(k, xi, make_float3(Fd[o + 0], Fd[o + 1], Fd[o + 2]), Ft + o, s, d);
        }
        const double2 SD = block_sum2(s, d, sh);
        if (threadIdx.x == 0) partials[(size_t)j * gridDim.x + blockIdx.x] = SD;
    }
    if (!fused) return;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&st->blocks_done, 1u) == gridDim.x * gridDim.y - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const long long n0 = st->step;
    const int Kw = min(K, keff);
    logu_fill(C, cf, n0, Kw);
    commit_decide(C, Kw, partials, gridDim.x, st->target_step - n0);
    if (stage_continues(C, Kw, K, staged, st->target_step - n0)) {
        if (threadIdx.x == 0) {
            st->blocks_done = 0u;
            st->stages += 1;
            stage_signal(next);
        }
        return;
    }
    commit_atoms(C, N, cf, species, w_qmid, w_pdraft, Fd, Ft, Fraw, ec_dF, ec_on, q, p, p_obabo, n0, 0, N);
    __syncthreads();
    if (threadIdx.x == 0) st->blocks_done = 0u;
    commit_stats(C, Kw, st, n0, K);
}

// A barrier over the whole grid of a cooperative launch (every block resident):
// each block's thread 0 arrives on the barrier's counter; the last arrival
// resets it and opens the next generation, for which the others wait (giving
// up after about two seconds).  Any grid size, launch after launch: a window
// verified in stages reduces a different number of steps per stage.
__device__ bool grid_sync_bounded(unsigned *cnt, unsigned *gen, unsigned total) {
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned g0;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(g0) : "l"(gen) : "memory");
        __threadfence();
        int ok = 1;
        if (atomicAdd(cnt, 1u) == total - 1u) {
            atomicExch(cnt, 0u);
            __threadfence();
            atomicAdd(gen, 1u);
        } else {
            const long long t0 = clock64();
            for (;;) {
                unsigned v;
                asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(gen) : "memory");
                if (v != g0) break;
                if (clock64() - t0 > 4000000000ll) {
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

// The whole transport in one cooperative launch: block (b, j) sums chunk b of
// window step j; after a grid barrier every block takes the decision (the same
// partials in the same order, so the same result) and commits its own slice of
// atoms, and block 0 updates the statistics.  The commit's FP64 work is spread
// over all nb*K SMs instead of one.
__global__ void __launch_bounds__(kTransThreads)
    transport_coop_kernel(int K, Geo g, Coef cf, const int *__restrict__ species, const float *__restrict__ Fd,
                          const float *__restrict__ Ft, DevState *__restrict__ st, double2 *__restrict__ partials,
                          const int *__restrict__ keff_p, int atoms_per_block, const double *__restrict__ w_qmid,
                          const double *__restrict__ w_pdraft, const float *__restrict__ Fraw,
                          float *__restrict__ ec_dF, int ec_on, double *__restrict__ q, double *__restrict__ p,
                          double *__restrict__ p_obabo, int j0, int staged, cudaGraphConditionalHandle next) {
    __shared__ double2 sh[32];
    __shared__ CommitShared C;
    // The run state and the draft's forces and noise come from kernels that
    // finished before the force gather began: read and drawn (with log u)
    // before the wait (block 0 rewrites the run state only after the grid
    // barrier).
    pdl_release();
    const volatile DevState *vs = st;
    const long long n0 = vs->step, tgt = vs->target_step;
    const int keff = *(const volatile int *)keff_p;
    if (n0 >= tgt) return;   // uniform over the grid
    const int N = g.N;
    const int j = j0 + blockIdx.y, nb = gridDim.x;   // window steps j0 .. K - 1
    const int a0 = blockIdx.x * atoms_per_block, a1 = min(N, a0 + atoms_per_block);
    constexpr int kPer = 4;   // atoms per thread held across the wait (chunks of up to 1024 atoms)
    float3 xi[kPer], fd[kPer];
    double kk[kPer];
    const unsigned long long n = (unsigned long long)(n0 + j + 1);
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
        const int i = a0 + threadIdx.x + u * (int)blockDim.x;
        xi[u] = fd[u] = make_float3(0.f, 0.f, 0.f);
        kk[u] = 0.0;
        if (j < keff && i < a1) {
            xi[u] = normals3(cf.seed, n, (uint32_t)i, 0u);
            kk[u] = species_pick(cf.aF_sig, species[i]);
            const size_t o = ((size_t)j * N + i) * 3;
            fd[u] = make_float3(Fd[o + 0], Fd[o + 1], Fd[o + 2]);
        }
    }
    // log u of every step (a long FP64 chain per thread), while the force gather finishes
    logu_fill(C, cf, n0, min(K, keff));
    pdl_wait();   // the target forces
    double s = 0.0, d = 0.0;
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
        const int i = a0 + threadIdx.x + u * (int)blockDim.x;
        if (j < keff && i < a1) atom_terms(kk[u], xi[u], fd[u], Ft + ((size_t)j * N + i) * 3, s, d);
    }
    const double2 SD = block_sum2(s, d, sh);
    if (threadIdx.x == 0 && j < keff) partials[(size_t)j * nb + blockIdx.x] = SD;
    if (!grid_sync_bounded(&st->grid_count, &st->grid_gen, (unsigned)(nb * gridDim.y))) {
        if (threadIdx.x == 0) atomicOr(&st->err, 16);
        return;
    }
    const int Kw = min(K, keff);
    commit_decide(C, Kw, partials, nb, tgt - n0);
    const int nblk = nb * gridDim.y, blk = blockIdx.y * nb + blockIdx.x;
    if (stage_continues(C, Kw, K, staged, tgt - n0)) {   // the same decision in every block
        if (blk == 0 && threadIdx.x == 0) {
            st->stages += 1;
            stage_signal(next);
        }
        return;
    }
    const int A = (N + nblk - 1) / nblk;
    commit_atoms(C, N, cf, species, w_qmid, w_pdraft, Fd, Ft, Fraw, ec_dF, ec_on, q, p, p_obabo, n0, blk * A,
                 min(N, blk * A + A));
    if (blk == 0) commit_stats(C, Kw, st, n0, K);
}

__global__ void __launch_bounds__(kTransThreads)
    transport_commit_kernel(int K, Geo g, Coef cf, const int *__restrict__ species, const double *__restrict__ w_qmid,
                            const double *__restrict__ w_pdraft, const float *__restrict__ Fd,
                            const float *__restrict__ Ft, const float *__restrict__ Fraw, float *__restrict__ ec_dF,
                            int ec_on, double *__restrict__ q, double *__restrict__ p,
                            double *__restrict__ p_obabo, DevState *__restrict__ st,
                            const double2 *__restrict__ partials, const int *__restrict__ keff_p, int n_part,
                            int atoms_per_block, int staged, cudaGraphConditionalHandle next) {
    __shared__ CommitShared C;
    __shared__ bool s_last;
    pdl_wait();
    pdl_release();
    if (st->step >= st->target_step) return;
    const int Kstage = K;
    K = min(K, *keff_p);   // the window holds the k_eff steps the draft reached
    const long long n0 = st->step;
    logu_fill(C, cf, n0, K);
    commit_decide(C, K, partials, n_part, st->target_step - n0);
    if (stage_continues(C, K, Kstage, staged, st->target_step - n0)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            st->stages += 1;
            stage_signal(next);
        }
        return;
    }
    const int a0 = blockIdx.x * atoms_per_block;
    commit_atoms(C, g.N, cf, species, w_qmid, w_pdraft, Fd, Ft, Fraw, ec_dF, ec_on, q, p, p_obabo, n0, a0,
                 min(g.N, a0 + atoms_per_block));
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&st->blocks_done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (threadIdx.x == 0) st->blocks_done = 0u;
    commit_stats(C, K, st, n0, Kstage);
}

void launch_transport_reduce(int K, const Geo &g, const Coef &cf, const int *species, const float *Fd,
                             const float *Ft, DevState *st, double2 *partials, const int *keff, cudaStream_t s,
                             int j0) {
    const int apb = transport_atoms_per_block(g.N);
    const int nb = (g.N + apb - 1) / apb;
    launch_dependent(transport_reduce_kernel, dim3(nb, K - j0), kTransThreads, 0, s, K, g, cf, species, Fd, Ft, st,
                     partials, keff, apb, 0, (const double *)nullptr, (const double *)nullptr, (const float *)nullptr,
                     (float *)nullptr, 0, (double *)nullptr, (double *)nullptr, (double *)nullptr, j0, 0,
                     (cudaGraphConditionalHandle)0);
}

void launch_transport_commit(int K, const Geo &g, const Coef &cf, const int *species, const double *w_qmid,
                             const double *w_pdraft, const float *Fd, const float *Ft, const float *Fraw, float *ec_dF,
                             int ec_on, double *q, double *p, double *p_obabo, DevState *st,
                             const double2 *partials, const int *keff, cudaStream_t s, int staged,
                             cudaGraphConditionalHandle next) {
    const int apb = transport_atoms_per_block(g.N);
    const int nb = (g.N + apb - 1) / apb;
    launch_dependent(transport_commit_kernel, nb, kTransThreads, 0, s, K, g, cf, species, w_qmid, w_pdraft, Fd, Ft,
                     Fraw, ec_dF, ec_on, q, p, p_obabo, st, (const double2 *)partials, keff, nb, apb, staged, next);
}

static int g_coop_blocks = -1;   // blocks of transport_coop_kernel the device keeps resident at once

cudaError_t transport_setup() {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, transport_coop_kernel, kTransThreads, 0);
    g_coop_blocks = e == cudaSuccess ? sms * per_sm : 0;
    return e;
}

// One cooperative launch when the grid fits on the device at once; else the
// one-block-per-step fused launch, or reduce then commit.
void launch_transport(int K, const Geo &g, const Coef &cf, const int *species, const double *w_qmid,
                      const double *w_pdraft, const float *Fd, const float *Ft, const float *Fraw, float *ec_dF,
                      int ec_on, double *q, double *p, double *p_obabo, DevState *st, double2 *partials,
                      const int *keff, cudaStream_t s, int j0, int staged, cudaGraphConditionalHandle next) {
    const int apb = transport_atoms_per_block(g.N);
    const int nb = (g.N + apb - 1) / apb;
    const int rows = K - j0;   // window steps reduced by this launch
    if (apb <= 4 * kTransThreads && nb * rows <= g_coop_blocks) {   // four atoms per thread at most
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(nb, rows);
        cfg.blockDim = dim3(kTransThreads);
        cfg.stream = s;
        cudaLaunchAttribute at[2];
        at[0].id = cudaLaunchAttributeCooperative;
        at[0].val.cooperative = 1;
        at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[1].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = at;
        cfg.numAttrs = pdl_enabled() ? 2 : 1;
        cudaLaunchKernelEx(&cfg, transport_coop_kernel, K, g, cf, species, Fd, Ft, st, partials, keff, apb, w_qmid,
                           w_pdraft, Fraw, ec_dF, ec_on, q, p, p_obabo, j0, staged, next);
        return;
    }
    if (nb == 1) {
        launch_dependent(transport_reduce_kernel, dim3(1, rows), kTransThreads, 0, s, K, g, cf, species, Fd, Ft, st,
                         partials, keff, apb, 1, w_qmid, w_pdraft, Fraw, ec_dF, ec_on, q, p, p_obabo, j0, staged,
                         next);
        return;
    }
    launch_transport_reduce(K, g, cf, species, Fd, Ft, st, partials, keff, s, j0);
    launch_transport_commit(K, g, cf, species, w_qmid, w_pdraft, Fd, Ft, Fraw, ec_dF, ec_on, q, p, p_obabo, st,
                            partials, keff, s, staged, next);
}

int transport_atoms_per_block(int N) {
    // at least one CTA per 1024 atoms, at most 148*4 CTAs per window step
    int apb = 1024;
    while ((N + apb - 1) / apb > 592 && apb < (1 << 20)) apb *= 2;
    return apb;
}

}  // namespace lsd
