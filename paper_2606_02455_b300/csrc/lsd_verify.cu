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
                                   const int *__restrict__ keff) {
    pdl_wait();
    pdl_release();
    const int row = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= M) return;
    const int N = g.N;
    const int j = row / N, i = row - j * N;
    if (keff && j >= *keff) {
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
// Per-warp staging of a row's descriptor neighbours in shared memory.
// ---------------------------------------------------------------------------
struct NbStage {
    float4 *g;   // (dx, dy, dz, 1/r): one 16-byte load per neighbour in the pair loops
    float4 *c;   // (fc, dfc, e1, e2)
    float *r;
    int *sp;
};

__device__ __forceinline__ NbStage nb_stage_ptrs(float *base, int cap) {
    NbStage s;   // cap is a multiple of 32: the float4 arrays stay 16-byte aligned
    s.g = reinterpret_cast<float4 *>(base);
    s.c = reinterpret_cast<float4 *>(base + 4 * cap);
    s.r = base + 8 * cap;
    s.sp = (int *)(base + 9 * cap);
    return s;
}
constexpr int kStageFloats = 10;

// The n (n - 1) / 2 unordered neighbour pairs of a row, flattened so that a
// warp's lanes stay busy whatever n is: pair t is (p, (p + d) mod n) with
// d = t / n + 1, p = t mod n (full diagonals d < n / 2, and for even n the
// half diagonal d = n / 2 with p < n / 2).  Within one diagonal the p are
// distinct and so are the q.  A lane starts at t = lane and advances by 32.
struct PairIter {
    int n, p, d;
    __device__ __forceinline__ PairIter(int n_, int lane) : n(n_), p(lane), d(1) {
        while (p >= n && n > 0) {
            p -= n;
            ++d;
        }
    }
    __device__ __forceinline__ int q() const { return p + d < n ? p + d : p + d - n; }
    __device__ __forceinline__ void next() {
        p += 32;
        while (p >= n) {
            p -= n;
            ++d;
        }
    }
};

__device__ __forceinline__ void nb_stage_load(const NbStage &S, const uint4 *fj, uint4 fi, const int *keys, int n,
                                              const Geo &g, float rc, int lane) {
    for (int p = lane; p < n; p += 32) {
        const int key = keys[p];
        const uint4 fk = fj[key >> 5];
        const float3 d = entry_disp(fi, fk, key & 31, g);
        const float r2 = dist2_rule(d.x, d.y, d.z);
        const float r = sqrtf(r2);
        float fc, dfc;
        cutoff_fn(r, rc, fc, dfc);
        S.g[p] = make_float4(d.x, d.y, d.z, 1.f / r);   // 1/r once per neighbour: the O(n^2) pair loops multiply
        S.c[p] = make_float4(fc, dfc, expf(-0.005f * r2), expf(-0.05f * r2));
        S.r[p] = r;
        S.sp[p] = (int)fk.w;
    }
    __syncwarp();
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
    NbStage S = nb_stage_ptrs(smem + (size_t)wib * kStageFloats * cap, cap);
    const int n = n_near[row];
    nb_stage_load(S, fj, fi, near_keys + (size_t)row * cap, n, g, P.desc_rc, lane);
    float *x = X + (size_t)row * P.d0p;
    const int nr = P.n_rbf;
    // radial
    {
        float acc[kMaxSpecies];
#pragma unroll
        for (int s = 0; s < kMaxSpecies; ++s) acc[s] = 0.f;
        const int kb = lane & 15;
        if (kb < nr) {
            const float mu = (float)kb * P.rbf_w;
            for (int p = lane >> 4; p < n; p += 2) {
                const float t = S.r[p] - mu;
                const float v = expf(-t * t * P.rbf_inv2w2) * S.c[p].x;
                const int sp = S.sp[p];
#pragma unroll
                for (int s = 0; s < kMaxSpecies; ++s) acc[s] += (sp == s) ? v : 0.f;
            }
        }
#pragma unroll
        for (int s = 0; s < kMaxSpecies; ++s) acc[s] += __shfl_down_sync(0xffffffffu, acc[s], 16);
        if (lane < nr)
            for (int s = 0; s < g.S; ++s) x[s * nr + lane] = acc[s];
    }
    // angular
    if (P.n_ang) {
        float a[kNAng];
#pragma unroll
        for (int t = 0; t < kNAng; ++t) a[t] = 0.f;
        const int npairs = n * (n - 1) / 2;
        PairIter it(n, lane);
        for (int t = lane; t < npairs; t += 32, it.next()) {
            const int p = it.p, q = it.q();
            {
                const float4 gp = S.g[p], gq = S.g[q], cp = S.c[p], cq = S.c[q];
                const float c = (gp.x * gq.x + gp.y * gq.y + gp.z * gq.z) * (gp.w * gq.w);
                const float ff = cp.x * cq.x;
                const float E1 = cp.z * cq.z * ff, E2 = cp.w * cq.w * ff;
                const float bp1 = 1.f + c, bm1 = 1.f - c;
                const float bp2 = bp1 * bp1, bm2 = bm1 * bm1, bp4 = bp2 * bp2, bm4 = bm2 * bm2;
                const float bp8 = bp4 * bp4, bm8 = bm4 * bm4;
                // zeta = 1 (2^0), 2 (2^-1), 4 (2^-3), 8 (2^-7)
                a[0] += bp1 * E1; a[1] += bp1 * E2; a[2] += bm1 * E1; a[3] += bm1 * E2;
                a[4] += 0.5f * bp2 * E1; a[5] += 0.5f * bp2 * E2; a[6] += 0.5f * bm2 * E1; a[7] += 0.5f * bm2 * E2;
                a[8] += 0.125f * bp4 * E1; a[9] += 0.125f * bp4 * E2; a[10] += 0.125f * bm4 * E1; a[11] += 0.125f * bm4 * E2;
                a[12] += 0.0078125f * bp8 * E1; a[13] += 0.0078125f * bp8 * E2;
                a[14] += 0.0078125f * bm8 * E1; a[15] += 0.0078125f * bm8 * E2;
            }
        }
        // the sixteen warp sums as one reduce-scatter: at offsets 16, 8, 4, 2
        // each lane keeps the half of its partial sums its offset bit selects
        // and adds the partner's partials of that half; lanes 2f and 2f+1 end
        // with the total of feature f (62 shuffles and adds instead of 160)
        static_assert(kNAng == 16, "the reduce-scatter is laid out for 16 features");
#pragma unroll
        for (int m = kNAng; m > 1; m >>= 1) {
            const bool up = (lane & (m == 16 ? 16 : m == 8 ? 8 : m == 4 ? 4 : 2)) != 0;
            const int o = m == 16 ? 16 : m == 8 ? 8 : m == 4 ? 4 : 2;
#pragma unroll
            for (int t = 0; t < m / 2; ++t) {
                const float keep = up ? a[t + m / 2] : a[t], send = up ? a[t] : a[t + m / 2];
                a[t] = keep + __shfl_xor_sync(0xffffffffu, send, o);
            }
        }
        a[0] += __shfl_xor_sync(0xffffffffu, a[0], 1);
        if ((lane & 1) == 0) x[g.S * nr + (lane >> 1)] = a[0];
    }
    // one-hot and padding
    const int off = g.S * nr + P.n_ang;
    for (int f = off + lane; f < P.d0p; f += 32) x[f] = (f == off + (int)fi.w) ? 1.f : 0.f;
}

// ---------------------------------------------------------------------------
// Pair gradients g_p = dE_i / d(r_p) and LJ forces.
// ---------------------------------------------------------------------------
// The angular term T(c_pq, r_p, r_q) of one unordered pair: dT/dd_p =
// A d_q + B_p d_p is added to p's accumulators (a*), and dT/dd_q = A d_p +
// B_q d_q is returned for q.  wang: dE/dX of the angular features.
__device__ __forceinline__ float4 pair_terms(const NbStage &S, const float (&wang)[kNAng], int p, int q, float &ax,
                                             float &ay, float &az, float &ab) {
    const float4 gp = S.g[p], gq = S.g[q], cp = S.c[p], cq = S.c[q];
    const float xp = gp.x, yp = gp.y, zp = gp.z, xq = gq.x, yq = gq.y, zq = gq.z;
    const float rip = gp.w, riq = gq.w;
    const float inv_pq = rip * riq;
    const float cth = (xp * xq + yp * yq + zp * zq) * inv_pq;
    const float fp = cp.x, fq = cq.x;
    const float E1 = cp.z * cq.z, E2 = cp.w * cq.w;
    // (1 + lambda c)^zeta and zeta (1 + lambda c)^(zeta - 1), lambda = +1 (p) and -1 (m)
    const float bp1 = 1.f + cth, bm1 = 1.f - cth;
    const float bp2 = bp1 * bp1, bm2 = bm1 * bm1, bp4 = bp2 * bp2, bm4 = bm2 * bm2;
    const float bp8 = bp4 * bp4, bm8 = bm4 * bm4;
    const float bp3 = bp2 * bp1, bm3 = bm2 * bm1, bp7 = bp4 * bp3, bm7 = bm4 * bm3;
    // per eta: S0 = sum_a w_a pref pow (value weights), S1 = dS0/dc
    float S0_1 = 0.f, S0_2 = 0.f, S1_1 = 0.f, S1_2 = 0.f;
    // zeta 1: pref 1
    S0_1 += wang[0] * bp1 + wang[2] * bm1;  S0_2 += wang[1] * bp1 + wang[3] * bm1;
    S1_1 += wang[0] - wang[2];              S1_2 += wang[1] - wang[3];
    // zeta 2: pref 1/2, zeta*pow1*pref = b
    S0_1 += 0.5f * (wang[4] * bp2 + wang[6] * bm2);  S0_2 += 0.5f * (wang[5] * bp2 + wang[7] * bm2);
    S1_1 += wang[4] * bp1 - wang[6] * bm1;           S1_2 += wang[5] * bp1 - wang[7] * bm1;
    // zeta 4: pref 1/8, zeta*pow1*pref = b^3/2
    S0_1 += 0.125f * (wang[8] * bp4 + wang[10] * bm4);  S0_2 += 0.125f * (wang[9] * bp4 + wang[11] * bm4);
    S1_1 += 0.5f * (wang[8] * bp3 - wang[10] * bm3);    S1_2 += 0.5f * (wang[9] * bp3 - wang[11] * bm3);
    // zeta 8: pref 1/128, zeta*pow1*pref = b^7/16
    S0_1 += 0.0078125f * (wang[12] * bp8 + wang[14] * bm8);
    S0_2 += 0.0078125f * (wang[13] * bp8 + wang[15] * bm8);
    S1_1 += 0.0625f * (wang[12] * bp7 - wang[14] * bm7);
    S1_2 += 0.0625f * (wang[13] * bp7 - wang[15] * bm7);
    const float ffq = fp * fq;
    const float S1E = (S1_1 * E1 + S1_2 * E2) * ffq, S0E = S0_1 * E1 + S0_2 * E2;
    // d/dd_p: S1 E ff (d_q / (r_p r_q) - c d_p / r_p^2) - 2 eta S0 E ff d_p + S0 E dfc_p fc_q d_p / r_p
    const float A = S1E * inv_pq;
    const float Bc = -2.f * (0.005f * S0_1 * E1 + 0.05f * S0_2 * E2) * ffq;
    const float Bp = Bc - S1E * cth * (rip * rip) + S0E * cp.y * fq * rip;
    const float Bq = Bc - S1E * cth * (riq * riq) + S0E * fp * cq.y * riq;
    ax += A * xq;
    ay += A * yq;
    az += A * zq;
    ab += Bp;
    return make_float4(A * xp, A * yp, A * zp, Bq);
}

// SLOTS > 0: neighbours per lane (lane l owns p = l + 32 s); every row has at
// most 32 SLOTS of them, and rows with more than 32 run the angular pairs by
// diagonals: in diagonal d lane l evaluates (p, p + d mod n) for its own p,
// keeps the p side in registers and hands the q side over through shared
// memory to q's owner (within one diagonal the q are distinct, so no two lanes
// write the same slot).  SLOTS = 0, and rows of at most 32: the pairs are
// flattened over all 32 lanes and both sides go to shared accumulators.
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
    float *wbuf = smem + (size_t)warps * kStageFloats * cap + (size_t)wib * P.d0p;
    float4 *tb = reinterpret_cast<float4 *>(smem + (size_t)warps * (kStageFloats * cap + P.d0p)) + (size_t)wib * cap;
    NbStage S = nb_stage_ptrs(smem + (size_t)wib * kStageFloats * cap, cap);
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
        const int nr = P.n_rbf;
        float wang[kNAng];   // dE/dX of the angular features, in registers across the pair loop
#pragma unroll
        for (int t = 0; t < kNAng; ++t) wang[t] = wbuf[g.S * nr + t];
        constexpr int R = SLOTS > 0 ? SLOTS : 1;
        float ax[R], ay[R], az[R], ab[R];
#pragma unroll
        for (int s = 0; s < R; ++s) ax[s] = ay[s] = az[s] = ab[s] = 0.f;
        float *sx = reinterpret_cast<float *>(tb), *sy = sx + cap, *sz = sx + 2 * cap, *sb = sx + 3 * cap;
        const bool flat = SLOTS == 0 || n <= 32;
        if (P.n_ang && flat) {
            // the pairs flattened over all 32 lanes, both sides added to shared accumulators
            for (int p = lane; p < n; p += 32) sx[p] = sy[p] = sz[p] = sb[p] = 0.f;
            __syncwarp();
            const int npairs = n * (n - 1) / 2;
            PairIter it(n, lane);
            for (int t = lane; t < npairs; t += 32, it.next()) {
                const int p = it.p, q = it.q();
                float px = 0.f, py = 0.f, pz = 0.f, pb = 0.f;
                const float4 v = pair_terms(S, wang, p, q, px, py, pz, pb);
                atomicAdd(sx + p, px);
                atomicAdd(sy + p, py);
                atomicAdd(sz + p, pz);
                atomicAdd(sb + p, pb);
                atomicAdd(sx + q, v.x);
                atomicAdd(sy + q, v.y);
                atomicAdd(sz + q, v.z);
                atomicAdd(sb + q, v.w);
            }
            __syncwarp();
        } else if (P.n_ang) {
            // diagonals d = 1 .. n/2; for even n the last one holds n/2 pairs (p < d)
            for (int d = 1; 2 * d <= n; ++d) {
                const bool half = 2 * d == n;
#pragma unroll
                for (int s = 0; s < R; ++s) {
                    const int p = lane + 32 * s;
                    if (p < n && (!half || p < d)) {
                        const int q = p + d < n ? p + d : p + d - n;
                        tb[q] = pair_terms(S, wang, p, q, ax[s], ay[s], az[s], ab[s]);
                    }
                }
                __syncwarp();
#pragma unroll
                for (int s = 0; s < R; ++s) {
                    const int q = lane + 32 * s;
                    if (q < n && (!half || q >= d)) {
                        const float4 v = tb[q];
                        ax[s] += v.x;
                        ay[s] += v.y;
                        az[s] += v.z;
                        ab[s] += v.w;
                    }
                }
                __syncwarp();
            }
        }
        // per neighbour: the radial term, then the angular sums (registers, or the shared accumulators)
        auto finish = [&](int p, float bx, float by, float bz, float bw) {
            const float4 gp = S.g[p], cp = S.c[p];
            const float xp = gp.x, yp = gp.y, zp = gp.z, rp = S.r[p], fp = cp.x, dfp = cp.y;
            const float rip = gp.w;
            // radial: c = sum_k w_k g_k'(r)
            float c = 0.f;
            const float *wr = wbuf + S.sp[p] * nr;
            for (int k = 0; k < nr; ++k) {
                const float t = rp - (float)k * P.rbf_w;
                const float phi = expf(-t * t * P.rbf_inv2w2);
                c += wr[k] * phi * (-t * P.rbf_invw2 * fp + dfp);
            }
            const float gx = c * xp * rip + bx + bw * xp;
            const float gy = c * yp * rip + by + bw * yp;
            const float gz = c * zp * rip + bz + bw * zp;
            pair_g[(size_t)row * cap + p] = make_float4(gx, gy, gz, 0.f);
            fx += gx;
            fy += gy;
            fz += gz;
        };
        if (flat) {
            for (int p = lane; p < n; p += 32)
                if (P.n_ang) finish(p, sx[p], sy[p], sz[p], sb[p]);
                else finish(p, 0.f, 0.f, 0.f, 0.f);
        } else {
#pragma unroll
            for (int s = 0; s < R; ++s)
                if (lane + 32 * s < n) finish(lane + 32 * s, ax[s], ay[s], az[s], ab[s]);
        }
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
                        const int *keff) {
    const int threads = 256;
    const int blocks = (int)(((size_t)M * 32 + threads - 1) / threads);
    auto k = min_image_only(g, rmax2f) ? neigh_build_kernel<false, true> : neigh_build_kernel<false, false>;
    launch_dependent(k, blocks, threads, 0, s, fix, nullptr, nullptr, 0, M, g, rmax2f, near2f, cap_near, cap_far,
                     near_keys, far_keys, n_near, n_far, st, keff);
}

void launch_neigh_list(const uint4 *fix, const int *vlist, const int *vcount, int vcap, int M, const Geo &g,
                       float rmax2f, float near2f, int cap_near, int cap_far, int *near_keys, int *far_keys,
                       int *n_near, int *n_far, DevState *st, const int *keff, cudaStream_t s) {
    const int threads = 256;
    const int blocks = (int)(((size_t)M * 32 + threads - 1) / threads);
    auto k = min_image_only(g, rmax2f) ? neigh_build_kernel<true, true> : neigh_build_kernel<true, false>;
    launch_dependent(k, blocks, threads, 0, s, fix, vlist, vcount, vcap, M, g, rmax2f, near2f, cap_near, cap_far,
                     near_keys, far_keys, n_near, n_far, st, keff);
}

size_t desc_smem_bytes(int warps, int cap) { return (size_t)warps * kStageFloats * cap * sizeof(float); }

void launch_desc(const uint4 *fix, const int *near_keys, const int *n_near, int cap, int M, const Geo &g,
                 const PotDev &P, float *X, cudaStream_t s) {
    const int warps = 8;
    const size_t sm = desc_smem_bytes(warps, cap);
    launch_dependent(desc_kernel, (M + warps - 1) / warps, warps * 32, sm, s, fix, near_keys, n_near, cap, M, g, P, X);
}

void launch_pairgrad(const uint4 *fix, const int *near_keys, const int *n_near, const int *far_keys, const int *n_far,
                     int cap, int cap_far, int M, const Geo &g, const PotDev &P, const float *dEdX, float4 *pair_g,
                     float4 *Fpart, float *E_lj, cudaStream_t s) {
    const int warps = 8;
    const size_t sm = desc_smem_bytes(warps, cap) + (size_t)warps * (P.d0p + 4 * cap) * sizeof(float);
    // lists of at most 128 hold mostly rows of a few dozen neighbours: flattened pairs with a small register
    // footprint; longer lists run their large rows by diagonals
    auto k = cap <= 128 ? pairgrad_kernel<0> : (cap <= 256 ? pairgrad_kernel<8> : pairgrad_kernel<16>);
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
    cudaError_t e = cudaFuncSetAttribute(desc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
    if (e != cudaSuccess) return e;
    const void *pk[3] = {(const void *)pairgrad_kernel<0>, (const void *)pairgrad_kernel<8>,
                         (const void *)pairgrad_kernel<16>};
    for (const void *k : pk) {
        e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace lsd
