// lsd_draft.cu -- the serial draft of a window (Alg. 2 draft_step, K times):
//   q_mid = q + (dt/2) p/m                          (A)
//   F~ = draft(q_mid)                               (LJ, or LJ + learned MLP)
//   <p~> = c1 p + (1+c1)(dt/2) kappa (F~ + dF)      (BOB mean, Eq. 4; dF = EC cache)
//   p' = <p~> + sigma xi_n,  q' = q_mid + (dt/2) p'/m  (BOB draw, A)
// The K steps are inherently serial, so for systems that fit one SM the whole
// window runs in one persistent CTA (1024 threads, the atoms' fixed-point
// coordinates in shared memory, one warp per atom and lanes over partners),
// paying one launch instead of K.  FP64 is used only for the state updates,
// with explicit round-to-nearest intrinsics so q_mid is reproducible bit for
// bit.  The window arrays written here (q_mid, p', F~, fixed point) are what
// the batched verification reads.
#include "lsd_common.cuh"
#include "lsd_kernels.h"

namespace lsd {

constexpr int kDraftThreads = 1024;
constexpr int kDraftWarps = kDraftThreads / 32;
constexpr int kLearnCap = 96;   // per-warp staged neighbours of the learned draft

// Per-axis candidate images for the draft (same rule as the verification).
__device__ __forceinline__ void lj_pair_force(const PotDev &P, int pr, float dx, float dy, float dz, float d2,
                                              float &fx, float &fy, float &fz) {
    const float s2 = P.lj_sig2[pr] / d2;
    const float s6 = s2 * s2 * s2, s12 = s6 * s6;
    const float fr = -P.lj_eps24[pr] * (2.f * s12 - s6) / d2;
    fx += fr * dx;
    fy += fr * dy;
    fz += fr * dz;
}

// Learned draft: descriptors (radial only) + MLP with BF16 weights and
// activations, FP32 accumulation; writes dE/dx of atom i to g_out[d0p].
__device__ void learned_atom_grad(const PotDev &P, const Geo &g, const uint4 *sfix, int i, float *stage, float *xbuf,
                                  float *g_out) {
    const int lane = threadIdx.x & 31;
    const int N = g.N;
    const uint4 fi = sfix[i];
    float *sr = stage, *sfc = stage + kLearnCap;
    int *ssp = (int *)(stage + 2 * kLearnCap);
    // stage members within the descriptor cutoff (order does not matter for sums of per-lane slots)
    int cnt = 0;
    for (int base = 0; base < N; base += 32) {
        const int k = base + lane;
        unsigned m = 0u;
        AxisOpts ox, oy, oz;
        ox.n = oy.n = oz.n = 0;
        if (k < N) {
            const uint4 fk = sfix[k];
            ox = axis_opts(fi.x, fk.x, g.scale_f[0], P.desc_rc2f);
            oy = axis_opts(fi.y, fk.y, g.scale_f[1], P.desc_rc2f);
            oz = axis_opts(fi.z, fk.z, g.scale_f[2], P.desc_rc2f);
            for (int bz = 0; bz < oz.n; ++bz)
                for (int by = 0; by < oy.n; ++by)
                    for (int bx = 0; bx < ox.n; ++bx) {
                        if (k == i && ox.s[bx] == 0 && oy.s[by] == 0 && oz.s[bz] == 0) continue;
                        if (dist2_rule(ox.d[bx], oy.d[by], oz.d[bz]) < P.desc_rc2f) m |= 1u << (bx + 2 * by + 4 * bz);
                    }
        }
        const int nm = __popc(m);
        int sc = nm;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, sc, o);
            if (lane >= o) sc += t;
        }
        const int tot = __shfl_sync(0xffffffffu, sc, 31);
        int w = cnt + sc - nm;
        for (int c = 0; c < 8; ++c) {
            if (!(m & (1u << c))) continue;
            if (w < kLearnCap) {
                const float dx = ox.d[c & 1], dy = oy.d[(c >> 1) & 1], dz = oz.d[c >> 2];
                const float r = sqrtf(dist2_rule(dx, dy, dz));
                float fc, dfc;
                cutoff_fn(r, P.desc_rc, fc, dfc);
                sr[w] = r;
                sfc[w] = fc;
                ssp[w] = (int)sfix[k].w;
            }
            ++w;
        }
        cnt += tot;
    }
    __syncwarp();
    const int n = cnt < kLearnCap ? cnt : kLearnCap;
    // radial descriptors x[s*nr + k]
    const int nr = P.n_rbf;
    {
        float acc[kMaxSpecies];
#pragma unroll
        for (int s = 0; s < kMaxSpecies; ++s) acc[s] = 0.f;
        const int kb = lane & 15;
        if (kb < nr) {
            const float mu = (float)kb * P.rbf_w;
            for (int p = lane >> 4; p < n; p += 2) {
                const float t = sr[p] - mu;
                const float v = expf(-t * t * P.rbf_inv2w2) * sfc[p];
#pragma unroll
                for (int s = 0; s < kMaxSpecies; ++s) acc[s] += (ssp[p] == s) ? v : 0.f;
            }
        }
#pragma unroll
        for (int s = 0; s < kMaxSpecies; ++s) acc[s] += __shfl_down_sync(0xffffffffu, acc[s], 16);
        for (int f = lane; f < P.d0p; f += 32) xbuf[f] = 0.f;
        __syncwarp();
        if (lane < nr)
            for (int s = 0; s < g.S; ++s) xbuf[s * nr + lane] = acc[s];
        if (lane == 0) xbuf[g.S * nr + P.n_ang + (int)fi.w] = 1.f;
    }
    __syncwarp();
    // MLP, one hidden layer, lane = hidden unit (width <= 32), BF16 operands
    const int W = P.width;
    float gh = 0.f;
    if (lane < W) {
        float h = P.b[0][lane];
        const __nv_bfloat16 *w1 = P.Wn_bf[0] + (size_t)lane * P.d0p;
        for (int f = 0; f < P.d0; ++f)
            h = fmaf(__bfloat162float(w1[f]), __bfloat162float(__float2bfloat16(xbuf[f])), h);
        gh = __bfloat162float(P.wout_bf[lane]) * dsiluf_(h);   // linear head: dE/dy = 1
    }
    __syncwarp();
    // dE/dx_f = sum_unit W1[unit][f] g_unit
    for (int f = 0; f < P.d0p; ++f) {
        float v = (lane < W && f < P.d0) ? __bfloat162float(P.Wn_bf[0][(size_t)lane * P.d0p + f]) * gh : 0.f;
        v = warp_sum(v);
        if (lane == 0) g_out[f] = v;
    }
    __syncwarp();
}

template <bool LEARNED>
__global__ void __launch_bounds__(kDraftThreads)
    draft_window_small_kernel(int K, Geo g, PotDev P, Coef cf, const int *__restrict__ species,
                              const double *__restrict__ q_base, const double *__restrict__ p_base,
                              const float *__restrict__ ec_dF, int ec_on, const DevState *__restrict__ st,
                              double *__restrict__ w_qmid, double *__restrict__ w_pdraft, float *__restrict__ w_Fd,
                              float *__restrict__ w_Fraw, uint4 *__restrict__ w_fix) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int N = g.N;
    uint4 *sfix = (uint4 *)smraw;
    float4 *sF = (float4 *)(sfix + N);
    float *sG = (float *)(sF + N);                                // learned: [N][d0p]
    float *sStage = sG + (LEARNED ? (size_t)N * P.d0p : 0);       // learned: per warp 3*cap + d0p
    if (st->step >= st->target_step) return;
    const long long n0 = st->step;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const size_t D = (size_t)3 * N;
    const float rc2_all = LEARNED ? fmaxf(P.lj_rc2f, P.desc_rc2f) : P.lj_rc2f;
    for (int j = 0; j < K; ++j) {
        // A: half-step positions and their fixed point
        for (int i = tid; i < N; i += kDraftThreads) {
            const int sp = species[i];
            const double hm = cf.hm[sp];
            uint32_t u[3];
            for (int c = 0; c < 3; ++c) {
                double qv, pv;
                if (j == 0) {
                    qv = q_base[3 * i + c];
                    pv = p_base[3 * i + c];
                } else {
                    const size_t o = (size_t)(j - 1) * D + 3 * i + c;
                    pv = w_pdraft[o];
                    qv = __dadd_rn(w_qmid[o], __dmul_rn(pv, hm));
                }
                const double qm = __dadd_rn(qv, __dmul_rn(pv, hm));
                w_qmid[(size_t)j * D + 3 * i + c] = qm;
                u[c] = fixpoint(qm, g.scale[c]);
            }
            const uint4 f = make_uint4(u[0], u[1], u[2], (unsigned)sp);
            sfix[i] = f;
            w_fix[(size_t)j * N + i] = f;
        }
        __syncthreads();
        if (LEARNED) {
            float *stage = sStage + (size_t)warp * (3 * kLearnCap + P.d0p);
            for (int i = warp; i < N; i += kDraftWarps)
                learned_atom_grad(P, g, sfix, i, stage, stage + 3 * kLearnCap, sG + (size_t)i * P.d0p);
            __syncthreads();
        }
        // forces: one warp per atom, lanes over partners
        for (int i = warp; i < N; i += kDraftWarps) {
            const uint4 fi = sfix[i];
            const int si = (int)fi.w;
            float fx = 0.f, fy = 0.f, fz = 0.f;
            for (int k = lane; k < N; k += 32) {
                const uint4 fk = sfix[k];
                const AxisOpts ox = axis_opts(fi.x, fk.x, g.scale_f[0], rc2_all);
                if (!ox.n) continue;
                const AxisOpts oy = axis_opts(fi.y, fk.y, g.scale_f[1], rc2_all);
                if (!oy.n) continue;
                const AxisOpts oz = axis_opts(fi.z, fk.z, g.scale_f[2], rc2_all);
                const int pr = si * g.S + (int)fk.w;
                for (int bz = 0; bz < oz.n; ++bz)
                    for (int by = 0; by < oy.n; ++by)
                        for (int bx = 0; bx < ox.n; ++bx) {
                            if (k == i && ox.s[bx] == 0 && oy.s[by] == 0 && oz.s[bz] == 0) continue;
                            const float dx = ox.d[bx], dy = oy.d[by], dz = oz.d[bz];
                            const float d2 = dist2_rule(dx, dy, dz);
                            if (P.has_lj && d2 < P.lj_rc2f) lj_pair_force(P, pr, dx, dy, dz, d2, fx, fy, fz);
                            if (LEARNED && d2 < P.desc_rc2f) {
                                // radial adjoint in gather form: (c_ik + c_ki) d/r
                                const float r = sqrtf(d2);
                                float fc, dfc;
                                cutoff_fn(r, P.desc_rc, fc, dfc);
                                const float *gi = sG + (size_t)i * P.d0p + (int)fk.w * P.n_rbf;
                                const float *gk = sG + (size_t)k * P.d0p + si * P.n_rbf;
                                float c = 0.f;
                                for (int b = 0; b < P.n_rbf; ++b) {
                                    const float t = r - (float)b * P.rbf_w;
                                    const float dg = expf(-t * t * P.rbf_inv2w2) * (-t * P.rbf_invw2 * fc + dfc);
                                    c += (gi[b] + gk[b]) * dg;
                                }
                                fx += c * dx / r;
                                fy += c * dy / r;
                                fz += c * dz / r;
                            }
                        }
            }
            fx = warp_sum(fx);
            fy = warp_sum(fy);
            fz = warp_sum(fz);
            if (lane == 0) sF[i] = make_float4(fx, fy, fz, 0.f);
        }
        __syncthreads();
        // BOB + A
        const unsigned long long n = (unsigned long long)(n0 + j + 1);
        for (int i = tid; i < N; i += kDraftThreads) {
            const int sp = species[i];
            const float4 F = sF[i];
            const float fr[3] = {F.x, F.y, F.z};
            const float3 xi3 = normals3(cf.seed, n, (uint32_t)i, 0u);
            const float xi[3] = {xi3.x, xi3.y, xi3.z};
            for (int c = 0; c < 3; ++c) {
                const size_t o = (size_t)j * D + 3 * i + c;
                const double pv = (j == 0) ? p_base[3 * i + c] : w_pdraft[o - D];
                const float fu = ec_on ? fr[c] + ec_dF[3 * i + c] : fr[c];
                const double mu = __dadd_rn(__dmul_rn(cf.c1, pv), __dmul_rn(cf.aF, (double)fu));
                w_pdraft[o] = __dadd_rn(mu, __dmul_rn(cf.sig[sp], (double)xi[c]));
                w_Fd[o] = fu;
                if (ec_on) w_Fraw[o] = fr[c];
            }
        }
        __syncthreads();
    }
}

size_t draft_small_smem_bytes(int N, const PotDev &P, bool learned) {
    size_t b = (size_t)N * (sizeof(uint4) + sizeof(float4));
    if (learned) b += ((size_t)N * P.d0p + (size_t)kDraftWarps * (3 * kLearnCap + P.d0p)) * sizeof(float);
    return b;
}

void launch_draft_small(bool learned, int K, const Geo &g, const PotDev &P, const Coef &cf, const int *species,
                        const double *q, const double *p, const float *ec_dF, int ec_on, const DevState *st,
                        double *w_qmid, double *w_pdraft, float *w_Fd, float *w_Fraw, uint4 *w_fix, cudaStream_t s) {
    const size_t sm = draft_small_smem_bytes(g.N, P, learned);
    if (learned)
        draft_window_small_kernel<true><<<1, kDraftThreads, sm, s>>>(K, g, P, cf, species, q, p, ec_dF, ec_on, st,
                                                                     w_qmid, w_pdraft, w_Fd, w_Fraw, w_fix);
    else
        draft_window_small_kernel<false><<<1, kDraftThreads, sm, s>>>(K, g, P, cf, species, q, p, ec_dF, ec_on, st,
                                                                      w_qmid, w_pdraft, w_Fd, w_Fraw, w_fix);
}

cudaError_t draft_kernels_setup(int max_smem) {
    cudaError_t e = cudaFuncSetAttribute(draft_window_small_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         max_smem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(draft_window_small_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                max_smem);
}

// ---------------------------------------------------------------------------
// Plain target ABOBA (the baseline): half step before the batched force
// evaluation, BOB + A after it.  Multi-CTA; the last CTA advances the step.
// ---------------------------------------------------------------------------
__global__ void plain_half_kernel(Geo g, Coef cf, const int *__restrict__ species, const double *__restrict__ q,
                                  const double *__restrict__ p, const DevState *__restrict__ st,
                                  double *__restrict__ qmid, uint4 *__restrict__ fix) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (st->step >= st->target_step || i >= g.N) return;
    const int sp = species[i];
    const double hm = cf.hm[sp];
    uint32_t u[3];
    for (int c = 0; c < 3; ++c) {
        const double qm = __dadd_rn(q[3 * i + c], __dmul_rn(p[3 * i + c], hm));
        qmid[3 * i + c] = qm;
        u[c] = fixpoint(qm, g.scale[c]);
    }
    fix[i] = make_uint4(u[0], u[1], u[2], (unsigned)sp);
}

__global__ void plain_finish_kernel(Geo g, Coef cf, const int *__restrict__ species, const double *__restrict__ qmid,
                                    const float *__restrict__ F, double *__restrict__ q, double *__restrict__ p,
                                    DevState *__restrict__ st) {
    __shared__ bool s_last;
    if (st->step >= st->target_step) return;
    const long long n0 = st->step;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < g.N) {
        const int sp = species[i];
        const float3 xi3 = normals3(cf.seed, (unsigned long long)(n0 + 1), (uint32_t)i, 0u);
        const float xi[3] = {xi3.x, xi3.y, xi3.z};
        for (int c = 0; c < 3; ++c) {
            const int o = 3 * i + c;
            const double mu = __dadd_rn(__dmul_rn(cf.c1, p[o]), __dmul_rn(cf.aF, (double)F[o]));
            const double pn = __dadd_rn(mu, __dmul_rn(cf.sig[sp], (double)xi[c]));
            p[o] = pn;
            q[o] = __dadd_rn(qmid[o], __dmul_rn(pn, cf.hm[sp]));
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
                       const DevState *st, double *qmid, uint4 *fix, cudaStream_t s) {
    plain_half_kernel<<<(g.N + 255) / 256, 256, 0, s>>>(g, cf, species, q, p, st, qmid, fix);
}

void launch_plain_finish(const Geo &g, const Coef &cf, const int *species, const double *qmid, const float *F,
                         double *q, double *p, DevState *st, cudaStream_t s) {
    plain_finish_kernel<<<(g.N + 255) / 256, 256, 0, s>>>(g, cf, species, qmid, F, q, p, st);
}

}  // namespace lsd
