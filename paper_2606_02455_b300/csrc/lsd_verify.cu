// lsd_verify.cu -- batched target force evaluation over a whole window
// (Alg. 2 verify_step's TargetModel.get_forces, run on all K*N atoms at once).
//
// Rows are (window step j, atom i), row = j*N + i.  Per row:
//   neigh_build_kernel   canonical neighbour lists (descriptor cutoff part and
//                        the rest up to the LJ cutoff), packed (k << 5 | code)
//   desc_kernel          radial + angular descriptors X[row][d0p]
//   (lsd_mlp.cu)         per-atom MLP energy and dE/dX
//   pairgrad_kernel      g_p = dE_i/d(r_p) for every descriptor neighbour p,
//                        its sum, and the LJ pair forces
//   force_gather_kernel  F_i = sum_p g_{i,p} - sum_p g_{k_p, rev(p)} + F_LJ,
//                        rev(p) found by binary search in the sorted list of k_p
// Everything is a gather in a fixed order: forces are bitwise deterministic.
#include <cmath>

#include "lsd_common.cuh"
#include "lsd_kernels.h"
#include "lsd_moments.cuh"
#include "lsd_pairs.cuh"

namespace lsd {

// ---------------------------------------------------------------------------
// Neighbour lists: one warp per row, all candidate atoms of the same window
// step, lanes over candidates.  Members of one candidate are kept in shift
// code order and lanes are compacted in order, so each row comes out sorted
// by (k, code) without a sort.
// ---------------------------------------------------------------------------
// LIST = false: candidates are all atoms of the window step (any configuration);
// LIST = true: candidates are the atom's sorted Verlet list.  With keff (the
// window paths) rows of window steps the draft did not reach (j >= k_eff) are
// left empty; without it (explicit configurations) every row is built.
// MINIMG (the cutoff below 0.499 of every box side): only the minimum image
// of a candidate can pass the rule (any other image along an axis is at least
// L/2, less rounding, away), and an atom's own images are beyond the cutoff, so
// each candidate gives at most one entry, with shift -k per axis.
template <bool LIST, bool MINIMG>
__global__ void neigh_build_kernel(const uint4 *__restrict__ fix, const int *__restrict__ vlist,
                                   const int *__restrict__ vcount, int vcap, int M, Geo g, float rmax2f, float near2f,
                                   int cap_near, int cap_far, int *__restrict__ near_keys, int *__restrict__ far_keys,
                                   int *__restrict__ n_near, int *__restrict__ n_far, DevState *st,
                                   const int *__restrict__ keff, int j_off) {
    pdl_wait();
    pdl_release();
    const int row = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= M) return;
    const int N = g.N;
    const int j = row / N, i = row - j * N;
    if (keff && j + j_off >= *keff) {   // j_off: the window step of row block 0 (a window verified in stages)
        if (lane == 0) {
            n_near[row] = 0;
            n_far[row] = 0;
        }
        return;
    }
    const uint4 *fj = fix + (size_t)j * N;
    const uint4 fi = fj[i];
    int *nk = near_keys + (size_t)row * cap_near;
    int *fk = far_keys + (size_t)row * cap_far;
    const int *cand = LIST ? vlist + (size_t)i * vcap : nullptr;
    const int ncand = LIST ? vcount[i] : N;
    int cn = 0, cf = 0;
    if (MINIMG) {
        const unsigned below = (1u << lane) - 1u;
        constexpr int kBatch = 8;   // candidates' positions loaded together: one memory latency per 8 passes
        for (int base0 = 0; base0 < ncand; base0 += 32 * kBatch) {
            int kk[kBatch];
            uint4 ff[kBatch];
#pragma unroll
            for (int u = 0; u < kBatch; ++u) {
                const int t = base0 + 32 * u + lane;
                kk[u] = LIST ? (t < ncand ? cand[t] : N) : (t < ncand ? t : N);
            }
#pragma unroll
            for (int u = 0; u < kBatch; ++u) ff[u] = kk[u] < N ? fj[kk[u]] : fi;
#pragma unroll
            for (int u = 0; u < kBatch; ++u) {
            if (base0 + 32 * u >= ncand) break;
            const int k = kk[u];
            bool in_n = false, in_f = false;
            int key = 0;
            if (k < N && k != i) {
                const uint4 fkk = ff[u];
                float dx, dy, dz;
                int kx, ky, kz;
                axis_min(fi.x, fkk.x, g.scale_f[0], dx, kx);
                axis_min(fi.y, fkk.y, g.scale_f[1], dy, ky);
                axis_min(fi.z, fkk.z, g.scale_f[2], dz, kz);
                const float d2 = dist2_rule(dx, dy, dz);
                in_n = d2 < rmax2f && d2 < near2f;
                in_f = d2 < rmax2f && !(d2 < near2f);
                key = (k << 5) | shift_code(-kx, -ky, -kz);
            }
            const unsigned bn = __ballot_sync(0xffffffffu, in_n), bf = __ballot_sync(0xffffffffu, in_f);
            const int wn = cn + __popc(bn & below), wf = cf + __popc(bf & below);
            if (in_n && wn < cap_near) nk[wn] = key;
            if (in_f && wf < cap_far) fk[wf] = key;
            cn += __popc(bn);
            cf += __popc(bf);
            }
        }
    }
    for (int base = 0; base < (MINIMG ? 0 : ncand); base += 32) {
        const int t = base + lane;
        const int k = LIST ? (t < ncand ? cand[t] : N) : t;
        unsigned mn = 0u, mf = 0u;
        AxisOpts ox, oy, oz;
        ox = oy = oz = AxisOpts{0.f, 0.f, 0, 0, 0};
        if (k < N) {
            const uint4 fkk = fj[k];
            ox = axis_opts(fi.x, fkk.x, g.scale_f[0], g.Lf[0], rmax2f);
            oy = axis_opts(fi.y, fkk.y, g.scale_f[1], g.Lf[1], rmax2f);
            oz = axis_opts(fi.z, fkk.z, g.scale_f[2], g.Lf[2], rmax2f);
            for (int bz = 0; bz < oz.n; ++bz)
                for (int by = 0; by < oy.n; ++by)
                    for (int bx = 0; bx < ox.n; ++bx) {
                        if (k == i && opt_s(ox, bx) == 0 && opt_s(oy, by) == 0 && opt_s(oz, bz) == 0) continue;
                        const float d2 = dist2_rule(opt_d(ox, bx), opt_d(oy, by), opt_d(oz, bz));
                        const unsigned bit = 1u << (bx + 2 * by + 4 * bz);
                        if (d2 < rmax2f) {
                            if (d2 < near2f) mn |= bit;
                            else mf |= bit;
                        }
                    }
        }
        const int nn = __popc(mn), nf = __popc(mf);
        int sn = nn, sf = nf;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int tn = __shfl_up_sync(0xffffffffu, sn, o);
            const int tf = __shfl_up_sync(0xffffffffu, sf, o);
            if (lane >= o) { sn += tn; sf += tf; }
        }
        const int tot_n = __shfl_sync(0xffffffffu, sn, 31), tot_f = __shfl_sync(0xffffffffu, sf, 31);
        int wn = cn + sn - nn, wf = cf + sf - nf;
        for (int c = 0; c < 8; ++c) {
            const unsigned bit = 1u << c;
            if (!((mn | mf) & bit)) continue;
            const int bx = c & 1, by = (c >> 1) & 1, bz = c >> 2;
            const int key = (k << 5) | shift_code(opt_s(ox, bx), opt_s(oy, by), opt_s(oz, bz));
            if (mn & bit) {
                if (wn < cap_near) nk[wn] = key;
                ++wn;
            } else {
                if (wf < cap_far) fk[wf] = key;
                ++wf;
            }
        }
        cn += tot_n;
        cf += tot_f;
    }
    if (lane == 0) {
        n_near[row] = cn < cap_near ? cn : cap_near;
        n_far[row] = cf < cap_far ? cf : cap_far;
        if (cn > cap_near || cf > cap_far) atomicOr(&st->err, 1);
    }
}

// ---------------------------------------------------------------------------
// Descriptors: radial by lanes over basis functions (two halves over
// neighbours), angular by lanes over neighbour pairs, warp reductions.
// ---------------------------------------------------------------------------
__global__ void desc_kernel(const uint4 *__restrict__ fix, const int *__restrict__ near_keys,
                            const int *__restrict__ n_near, int cap, int M, Geo g, PotDev P, float *__restrict__ X) {
    pdl_wait();
    pdl_release();
    extern __shared__ __align__(16) float smem[];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row = blockIdx.x * (blockDim.x >> 5) + wib;
    if (row >= M) return;
    const int N = g.N;
    const int j = row / N, i = row - j * N;
    const uint4 *fj = fix + (size_t)j * N;
    const uint4 fi = fj[i];
    NbStage S = nb_stage_ptrs(smem + (size_t)wib * kNbStageFloats * cap, cap);
    const int n = n_near[row];
    nb_stage_load(S, fj, fi, near_keys + (size_t)row * cap, n, g, P.desc_rc, lane);
    desc_row(S, n, P, g.S, (int)fi.w, X + (size_t)row * P.d0p, lane);
}

// The same descriptors with the angular block by moments (lsd_moments.cuh),
// the row's moments to mom [row][kMomFloats] for the adjoint.  Shared memory
// per warp: one chunk of 32 neighbours' staged powers and geometry (later the
// row's moments), 5 KB: four blocks of eight warps per SM.
__global__ void __launch_bounds__(256, 4) desc_mom_kernel(const uint4 *__restrict__ fix, const int *__restrict__ near_keys,
                                const int *__restrict__ n_near, int cap, int M, Geo g, PotDev P, float *__restrict__ X,
                                float *__restrict__ mom) {
    pdl_wait();
    pdl_release();
    extern __shared__ __align__(16) float smem[];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row = blockIdx.x * (blockDim.x >> 5) + wib;
    if (row >= M) return;
    const int N = g.N;
    const int j = row / N, i = row - j * N;
    const uint4 *fj = fix + (size_t)j * N;
    const uint4 fi = fj[i];
    float *tab = smem + (size_t)wib * kMomTabFloats;
    const int n = n_near[row];
    float *x = X + (size_t)row * P.d0p;
    mom_row_descriptors(fj, fi, near_keys + (size_t)row * cap, n, g, P, g.S, tab, mom + (size_t)row * kMomFloats, x,
                        lane);
    desc_onehot(P, g.S, (int)fi.w, x, lane);
}

// ---------------------------------------------------------------------------
// Pair gradients g_p = dE_i / d(r_p) and LJ forces.
// ---------------------------------------------------------------------------

// SLOTS: neighbours per lane (lane l owns p = l + 32 s); every row has at most
// 32 SLOTS of them.  The angular pairs run by diagonals (row_pair_grads): a
// fixed order of summation with no atomics, so the forces do not depend on the
// launch shape.
template <int SLOTS>
__global__ void pairgrad_kernel(const uint4 *__restrict__ fix, const int *__restrict__ near_keys,
                                const int *__restrict__ n_near, const int *__restrict__ far_keys,
                                const int *__restrict__ n_far, int cap, int cap_far, int M, Geo g, PotDev P,
                                const float *__restrict__ dEdX, float4 *__restrict__ pair_g,
                                float4 *__restrict__ Fpart, float *__restrict__ E_lj) {
    // MLP potentials: the previous kernel is the MLP, and the neighbour lists
    // and positions come from kernels that finished before it began, so the
    // geometry staging and the LJ part run before the wait, while the MLP still
    // runs; only dE/dX needs it.  Otherwise the lists come from the previous
    // kernel itself.
    if (!P.has_mlp) pdl_wait();
    pdl_release();
    extern __shared__ __align__(16) float smem[];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row = blockIdx.x * (blockDim.x >> 5) + wib;
    if (row >= M) return;
    const int N = g.N;
    const int j = row / N, i = row - j * N;
    const uint4 *fj = fix + (size_t)j * N;
    const uint4 fi = fj[i];
    const int warps = blockDim.x >> 5;
    float *wbuf = smem + (size_t)warps * kNbStageFloats * cap + (size_t)wib * P.d0p;
    float4 *tb = reinterpret_cast<float4 *>(smem + (size_t)warps * (kNbStageFloats * cap + P.d0p)) + (size_t)wib * cap;
    NbStage S = nb_stage_ptrs(smem + (size_t)wib * kNbStageFloats * cap, cap);
    const int n = n_near[row];
    const int *keys = near_keys + (size_t)row * cap;
    float fx = 0.f, fy = 0.f, fz = 0.f, e = 0.f;
    if (P.has_mlp) nb_stage_load(S, fj, fi, keys, n, g, P.desc_rc, lane);
    if (P.has_lj) {
        const int si = (int)fi.w;
        const int nf = n_far[row];
        const int *fkeys = far_keys + (size_t)row * cap_far;
        for (int t = lane; t < n + nf; t += 32) {
            const int key = t < n ? keys[t] : fkeys[t - n];
            const uint4 fk = fj[key >> 5];
            const float3 d = entry_disp(fi, fk, key & 31, g);
            const float d2 = dist2_rule(d.x, d.y, d.z);
            if (!(d2 < P.lj_rc2f)) continue;
            const int pr = si * g.S + (int)fk.w;
            const float s2 = P.lj_sig2[pr] / d2;
            const float s6 = s2 * s2 * s2, s12 = s6 * s6;
            const float fr = -P.lj_eps24[pr] * (2.f * s12 - s6) / d2;   // (dU/dr)/r
            fx += fr * d.x;
            fy += fr * d.y;
            fz += fr * d.z;
            e += 0.5f * (P.lj_eps4[pr] * (s12 - s6) - P.lj_shift[pr]);
        }
    }
    if (P.has_mlp) {
        pdl_wait();
        for (int f = lane; f < P.d0p; f += 32) wbuf[f] = dEdX[(size_t)row * P.d0p + f];
        __syncwarp();
        row_pair_grads<SLOTS>(S, n, P, g.S, wbuf, tb, pair_g + (size_t)row * cap, lane, fx, fy, fz);
    }
    fx = warp_sum(fx);
    fy = warp_sum(fy);
    fz = warp_sum(fz);
    e = warp_sum(e);
    if (lane == 0) {
        Fpart[row] = make_float4(fx, fy, fz, 0.f);
        E_lj[row] = e;
    }
}

// The pair gradients with the angular adjoint by moments (lsd_moments.cuh):
// lanes over neighbours throughout, each lane forming its neighbour's
// geometry in registers (the same operations as the descriptor staging), so
// only dE/dX and the adjoint coefficients live in shared memory.  LJ pairs of
// the descriptor list are taken in the same pass.
__global__ void __launch_bounds__(256, 4)
    pairgrad_mom_kernel(const uint4 *__restrict__ fix, const int *__restrict__ near_keys,
                        const int *__restrict__ n_near, const int *__restrict__ far_keys,
                        const int *__restrict__ n_far, int cap, int cap_far, int M, Geo g, PotDev P,
                        const float *__restrict__ dEdX, float4 *__restrict__ pair_g, float4 *__restrict__ Fpart,
                        float *__restrict__ E_lj, const float *__restrict__ mom) {
    pdl_release();
    extern __shared__ __align__(16) float smem[];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row = blockIdx.x * (blockDim.x >> 5) + wib;
    if (row >= M) return;
    const int N = g.N;
    const int j = row / N, i = row - j * N;
    const uint4 *fj = fix + (size_t)j * N;
    const uint4 fi = fj[i];
    const int si = (int)fi.w;
    float *wbuf = smem + (size_t)wib * (P.d0p + 2 * kMomLd + 32);
    float2 *psi = reinterpret_cast<float2 *>(wbuf + P.d0p);
    float *gk = wbuf + P.d0p + 2 * kMomLd;
    const int n = n_near[row];
    const int *keys = near_keys + (size_t)row * cap;
    float fx = 0.f, fy = 0.f, fz = 0.f, e = 0.f;
    auto lj_pair = [&](const float3 &d, float d2, int sk) {
        if (!(P.has_lj && d2 < P.lj_rc2f)) return;
        const int pr = si * g.S + sk;
        const float s2 = P.lj_sig2[pr] / d2;
        const float s6 = s2 * s2 * s2, s12 = s6 * s6;
        const float fr = -P.lj_eps24[pr] * (2.f * s12 - s6) / d2;   // (dU/dr)/r
        fx += fr * d.x;
        fy += fr * d.y;
        fz += fr * d.z;
        e += 0.5f * (P.lj_eps4[pr] * (s12 - s6) - P.lj_shift[pr]);
    };
    {
        // LJ partners beyond the descriptor cutoff, while the network still runs
        const int nf = n_far[row];
        const int *fkeys = far_keys + (size_t)row * cap_far;
        for (int t = lane; t < nf; t += 32) {
            const int key = fkeys[t];
            const uint4 fk = fj[key >> 5];
            const float3 d = entry_disp(fi, fk, key & 31, g);
            lj_pair(d, dist2_rule(d.x, d.y, d.z), (int)fk.w);
        }
    }
    pdl_wait();
    // the row's moments, loads issued before the coefficients they scale are formed
    constexpr int kPhiPerLane = (kMomFloats + 31) / 32;
    const float *mrow = mom + (size_t)row * kMomFloats;
    float phi[kPhiPerLane];
#pragma unroll
    for (int u = 0; u < kPhiPerLane; ++u) phi[u] = lane + 32 * u < kMomFloats ? __ldg(mrow + lane + 32 * u) : 0.f;
    for (int f = lane; f < P.d0p; f += 32) wbuf[f] = dEdX[(size_t)row * P.d0p + f];
    __syncwarp();
    mom_gamma_kappa(wbuf + g.S * P.n_rbf, gk, lane);
    float *psf = reinterpret_cast<float *>(psi);
#pragma unroll
    for (int u = 0; u < kPhiPerLane; ++u) {
        const int k = lane + 32 * u;
        const int et = k >= kMomLd ? 1 : 0, kk = k - et * kMomLd;
        if (k < kMomFloats && kk < kMomAlpha) {
            const float2 dm = kMomCoefTab.dm[kk];
            psf[2 * kk + et] = 2.f * dm.y * gk[et * (kMomDeg + 1) + (int)dm.x] * phi[u];
        }
    }
    __syncwarp();
    const float k1 = gk[2 * (kMomDeg + 1)], k2 = gk[2 * (kMomDeg + 1) + 1];
    const int nr = P.n_rbf;
    float4 *pg = pair_g + (size_t)row * cap;
    for (int p = lane; p < n; p += 32) {
        const int key = keys[p];
        const uint4 fk = fj[key >> 5];
        const float3 d = entry_disp(fi, fk, key & 31, g);
        const float r2 = dist2_rule(d.x, d.y, d.z);
        lj_pair(d, r2, (int)fk.w);
        if (!P.has_mlp) continue;
        const float r = sqrtf(r2);
        float fc, dfc;
        cutoff_fn(r, P.desc_rc, fc, dfc);
        const float ri = 1.f / r;
        const float e1 = expf(-0.005f * r2), e2 = expf(-0.05f * r2);
        // radial: c = sum_k w_k g_k'(r)
        float cr = 0.f;
        const float *wr = wbuf + (int)fk.w * nr;
        for (int k = 0; k < nr; ++k) {
            const float t = r - (float)k * P.rbf_w;
            const float ph = __expf(-t * t * P.rbf_inv2w2);   // as in desc_radial
            cr += wr[k] * ph * (-t * P.rbf_invw2 * fc + dfc);
        }
        const float ux = d.x * ri, uy = d.y * ri, uz = d.z * ri;
        float F[2], G[2][3];
        mom_eval(psi, ux, uy, uz, F, G);
        const float w1 = fc * e1, w2 = fc * e2;
        const float wp1 = (dfc - 2.f * 0.005f * r * fc) * e1, wp2 = (dfc - 2.f * 0.05f * r * fc) * e2;
        cr += (F[0] + 2.f * k1 * w1) * wp1 + (F[1] + 2.f * k2 * w2) * wp2;
        const float bx = w1 * G[0][0] + w2 * G[1][0], by = w1 * G[0][1] + w2 * G[1][1],
                    bz = w1 * G[0][2] + w2 * G[1][2];
        const float ub = ux * bx + uy * by + uz * bz;
        const float gx = cr * ux + (bx - ub * ux) * ri;
        const float gy = cr * uy + (by - ub * uy) * ri;
        const float gz = cr * uz + (bz - ub * uz) * ri;
        pg[p] = make_float4(gx, gy, gz, 0.f);
        fx += gx;
        fy += gy;
        fz += gz;
    }
    fx = warp_sum(fx);
    fy = warp_sum(fy);
    fz = warp_sum(fz);
    e = warp_sum(e);
    if (lane == 0) {
        Fpart[row] = make_float4(fx, fy, fz, 0.f);
        E_lj[row] = e;
    }
}

// ---------------------------------------------------------------------------
// F_i = Fpart_i - sum_p g[rev(p)]: the reverse entry (i, -s) is looked up by
// binary search in the (sorted) descriptor list of the neighbour's row.
// ---------------------------------------------------------------------------
__global__ void force_gather_kernel(const int *__restrict__ near_keys, const int *__restrict__ n_near, int cap, int M,
                                    int N, int has_mlp, const float4 *__restrict__ pair_g,
                                    const float4 *__restrict__ Fpart, const float *__restrict__ E_lj,
                                    const float *__restrict__ E_mlp, float *__restrict__ F_out,
                                    float *__restrict__ E_out, DevState *st) {
    // the lists come from a kernel that finished before the pair gradients
    // released this launch: the reverse entries are found before the wait
    pdl_release();
    const int row = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= M) return;
    const int j = row / N, i = row - j * N;
    constexpr int kSlots = 8;   // reverse entries held per lane across the wait (lists of up to 256)
    int at[kSlots];
    const int n = has_mlp ? n_near[row] : 0;
#pragma unroll
    for (int u = 0; u < kSlots; ++u) {
        const int p = lane + 32 * u;
        at[u] = p < n ? find_reverse(near_keys, n_near, cap, N, j, i, p, &st->err) : -1;
    }
    pdl_wait();
    float ax = 0.f, ay = 0.f, az = 0.f;
    if (has_mlp) {
#pragma unroll
        for (int u = 0; u < kSlots; ++u)
            if (at[u] >= 0) {
                const float4 gv = pair_g[at[u]];
                ax += gv.x;
                ay += gv.y;
                az += gv.z;
            }
        for (int p = lane + 32 * kSlots; p < n; p += 32) {
            const int a = find_reverse(near_keys, n_near, cap, N, j, i, p, &st->err);
            if (a >= 0) {
                const float4 gv = pair_g[a];
                ax += gv.x;
                ay += gv.y;
                az += gv.z;
            }
        }
        ax = warp_sum(ax);
        ay = warp_sum(ay);
        az = warp_sum(az);
    }
    if (lane == 0) {
        const float4 fp = Fpart[row];
        F_out[(size_t)row * 3 + 0] = fp.x - ax;
        F_out[(size_t)row * 3 + 1] = fp.y - ay;
        F_out[(size_t)row * 3 + 2] = fp.z - az;
        if (E_out) E_out[row] = E_lj[row] + (has_mlp ? E_mlp[row] : 0.f);
    }
}

// ---------------------------------------------------------------------------
// Half-step positions for arbitrary configurations (used by the batched force
// entry points): fixed point of each row's position.
// ---------------------------------------------------------------------------
__global__ void fixpoint_kernel(const double *__restrict__ q, const int *__restrict__ species, int M, Geo g,
                                uint4 *__restrict__ fix) {
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= M) return;
    const int i = row % g.N;
    const double *qr = q + (size_t)row * 3;
    fix[row] = make_uint4(fixpoint(qr[0], g.scale[0]), fixpoint(qr[1], g.scale[1]), fixpoint(qr[2], g.scale[2]),
                          (unsigned)species[i]);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
void launch_fixpoint(const double *q, const int *species, int M, const Geo &g, uint4 *fix, cudaStream_t s) {
    fixpoint_kernel<<<(M + 255) / 256, 256, 0, s>>>(q, species, M, g, fix);
}

// rc < 0.499 min(L): the minimum-image form of the rule applies
static bool min_image_only(const Geo &g, float rmax2f) {
    const float lmin = fminf(g.Lf[0], fminf(g.Lf[1], g.Lf[2]));
    return std::sqrt((double)rmax2f) < 0.499 * (double)lmin;
}

void launch_neigh_build(const uint4 *fix, int M, const Geo &g, float rmax2f, float near2f, int cap_near, int cap_far,
                        int *near_keys, int *far_keys, int *n_near, int *n_far, DevState *st, cudaStream_t s,
                        const int *keff, int j_off) {
    const int threads = 256;
    const int blocks = (int)(((size_t)M * 32 + threads - 1) / threads);
    auto k = min_image_only(g, rmax2f) ? neigh_build_kernel<false, true> : neigh_build_kernel<false, false>;
    launch_dependent(k, blocks, threads, 0, s, fix, nullptr, nullptr, 0, M, g, rmax2f, near2f, cap_near, cap_far,
                     near_keys, far_keys, n_near, n_far, st, keff, j_off);
}

void launch_neigh_list(const uint4 *fix, const int *vlist, const int *vcount, int vcap, int M, const Geo &g,
                       float rmax2f, float near2f, int cap_near, int cap_far, int *near_keys, int *far_keys,
                       int *n_near, int *n_far, DevState *st, const int *keff, cudaStream_t s, int j_off) {
    const int threads = 256;
    const int blocks = (int)(((size_t)M * 32 + threads - 1) / threads);
    auto k = min_image_only(g, rmax2f) ? neigh_build_kernel<true, true> : neigh_build_kernel<true, false>;
    launch_dependent(k, blocks, threads, 0, s, fix, vlist, vcount, vcap, M, g, rmax2f, near2f, cap_near, cap_far,
                     near_keys, far_keys, n_near, n_far, st, keff, j_off);
}

size_t desc_smem_bytes(int warps, int cap) { return (size_t)warps * kNbStageFloats * cap * sizeof(float); }

void launch_desc(const uint4 *fix, const int *near_keys, const int *n_near, int cap, int M, const Geo &g,
                 const PotDev &P, float *X, cudaStream_t s, float *mom) {
    const int warps = 8;
    if (mom && P.n_ang) {
        const size_t sm = (size_t)warps * kMomTabFloats * sizeof(float);
        launch_dependent(desc_mom_kernel, (M + warps - 1) / warps, warps * 32, sm, s, fix, near_keys, n_near, cap, M,
                         g, P, X, mom);
        return;
    }
    const size_t sm = desc_smem_bytes(warps, cap);
    launch_dependent(desc_kernel, (M + warps - 1) / warps, warps * 32, sm, s, fix, near_keys, n_near, cap, M, g, P, X);
}

void launch_pairgrad(const uint4 *fix, const int *near_keys, const int *n_near, const int *far_keys, const int *n_far,
                     int cap, int cap_far, int M, const Geo &g, const PotDev &P, const float *dEdX, float4 *pair_g,
                     float4 *Fpart, float *E_lj, cudaStream_t s, const float *mom) {
    const int warps = 8;
    if (mom && P.n_ang && P.has_mlp) {
        const size_t sm = (size_t)warps * (P.d0p + 2 * kMomLd + 32) * sizeof(float);
        launch_dependent(pairgrad_mom_kernel, (M + warps - 1) / warps, warps * 32, sm, s, fix, near_keys, n_near,
                         far_keys, n_far, cap, cap_far, M, g, P, dEdX, pair_g, Fpart, E_lj, mom);
        return;
    }
    const size_t sm = desc_smem_bytes(warps, cap) + (size_t)warps * (P.d0p + 4 * cap) * sizeof(float);
    // lists of at most 128 hold mostly rows of a few dozen neighbours: flattened pairs with a small register
    // footprint; longer lists run their large rows by diagonals
    auto k = cap <= 128 ? pairgrad_kernel<4> : (cap <= 256 ? pairgrad_kernel<8> : pairgrad_kernel<16>);
    launch_dependent(k, (M + warps - 1) / warps, warps * 32, sm, s, fix, near_keys, n_near, far_keys, n_far, cap,
                     cap_far, M, g, P, dEdX, pair_g, Fpart, E_lj);
}

void launch_force_gather(const int *near_keys, const int *n_near, int cap, int M, int N, int has_mlp,
                         const float4 *pair_g, const float4 *Fpart, const float *E_lj, const float *E_mlp, float *F,
                         float *E_out, DevState *st, cudaStream_t s) {
    const int threads = 256;
    const int blocks = (int)(((size_t)M * 32 + threads - 1) / threads);
    launch_dependent(force_gather_kernel, blocks, threads, 0, s, near_keys, n_near, cap, M, N, has_mlp, pair_g, Fpart,
                     E_lj, E_mlp, F, E_out, st);
}

cudaError_t verify_kernels_setup(int max_smem) {
    static_assert(kMomRowFloats == kMomFloats, "moment row size");
    cudaError_t e = cudaFuncSetAttribute(desc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(desc_mom_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
    if (e != cudaSuccess) return e;
    const void *pk[4] = {(const void *)pairgrad_kernel<4>, (const void *)pairgrad_kernel<8>,
                         (const void *)pairgrad_kernel<16>, (const void *)pairgrad_mom_kernel};
    for (const void *k : pk) {
        e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace lsd
