// lsd_pairs.cuh -- device helpers of the descriptor and pair-gradient code,
// shared by the batched verification kernels (lsd_verify.cu) and the fused
// plain-target step (lsd_plain.cu): per-warp staging of a row's descriptor
// neighbours, the flattened enumeration of neighbour pairs, and the angular
// term of one pair with its gradient.
#pragma once

#include "lsd_common.cuh"

namespace lsd {

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
constexpr int kNbStageFloats = 10;

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


// The angular weights of one row in the packed form of the pair loop.  The
// sixteen angular features are T[z][l][e] = 2^(1 - zeta) sum_{p<q} (1 + lambda
// c)^zeta E_e fc_p fc_q (zeta = 1, 2, 4, 8 for z = 0..3, lambda = +1, -1 for
// l = 0, 1, eta = 0.005, 0.05 for e = 0, 1), feature index 4 z + 2 l + e.  With
// w = dE/dX of those features, the pair loop needs, per eta,
//   S0_e = sum_z pref_z (w[z][0][e] b+^zeta + w[z][1][e] b-^zeta)
//   S1_e = dS0_e/dc = sum_z zeta pref_z (w[z][0][e] b+^(zeta-1) - w[z][1][e] b-^(zeta-1))
// with b+- = 1 +- c.  Both are dot products over (z, lambda); packed over lambda
// they are fused multiply-adds of float pairs (two lanes of FP32 work per
// instruction) with the (b+^k, b-^k) pairs.
struct AngW {
    float2 w0[4][2];   // [z][e]: pref_z (w[z][0][e], w[z][1][e])
    float2 w1[3][2];   // [z - 1][e], zeta 2, 4, 8: zeta pref_z (w[z][0][e], -w[z][1][e])
    float c1[2];       // [e]: the zeta = 1 term of S1_e, w[0][0][e] - w[0][1][e]
};

__device__ __forceinline__ AngW ang_weights(const float (&w)[kNAng]) {
    constexpr float pref[4] = {1.f, 0.5f, 0.125f, 0.0078125f};   // 2^(1 - zeta)
    constexpr float zpref[4] = {1.f, 1.f, 0.5f, 0.0625f};         // zeta 2^(1 - zeta)
    AngW a;
#pragma unroll
    for (int z = 0; z < 4; ++z)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            a.w0[z][e] = make_float2(pref[z] * w[4 * z + e], pref[z] * w[4 * z + 2 + e]);
            if (z > 0) a.w1[z - 1][e] = make_float2(zpref[z] * w[4 * z + e], -zpref[z] * w[4 * z + 2 + e]);
        }
    a.c1[0] = w[0] - w[2];
    a.c1[1] = w[1] - w[3];
    return a;
}

// The angular term T(c_pq, r_p, r_q) of one unordered pair: dT/dd_p =
// A d_q + B_p d_p is added to p's accumulators (a*), and dT/dd_q = A d_p +
// B_q d_q is returned for q.
__device__ __forceinline__ float4 pair_terms(const NbStage &S, const AngW &W, int p, int q, float &ax, float &ay,
                                             float &az, float &ab) {
    const float4 gp = S.g[p], gq = S.g[q], cp = S.c[p], cq = S.c[q];
    const float xp = gp.x, yp = gp.y, zp = gp.z, xq = gq.x, yq = gq.y, zq = gq.z;
    const float rip = gp.w, riq = gq.w;
    const float inv_pq = rip * riq;
    const float cth = (xp * xq + yp * yq + zp * zq) * inv_pq;
    const float fp = cp.x, fq = cq.x;
    // (b+^k, b-^k) for k = 1, 2, 3, 4, 7, 8
    const float2 b1 = make_float2(1.f + cth, 1.f - cth);
    const float2 b2 = __fmul2_rn(b1, b1), b4 = __fmul2_rn(b2, b2);
    const float2 b3 = __fmul2_rn(b2, b1), b8 = __fmul2_rn(b4, b4), b7 = __fmul2_rn(b4, b3);
    float2 t0[2], t1[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        t0[e] = __fmul2_rn(W.w0[0][e], b1);
        t0[e] = __ffma2_rn(W.w0[1][e], b2, t0[e]);
        t0[e] = __ffma2_rn(W.w0[2][e], b4, t0[e]);
        t0[e] = __ffma2_rn(W.w0[3][e], b8, t0[e]);
        t1[e] = __ffma2_rn(W.w1[0][e], b1, make_float2(W.c1[e], 0.f));
        t1[e] = __ffma2_rn(W.w1[1][e], b3, t1[e]);
        t1[e] = __ffma2_rn(W.w1[2][e], b7, t1[e]);
    }
    const float S0_1 = t0[0].x + t0[0].y, S0_2 = t0[1].x + t0[1].y;
    const float S1_1 = t1[0].x + t1[0].y, S1_2 = t1[1].x + t1[1].y;
    const float E1 = cp.z * cq.z, E2 = cp.w * cq.w;
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

// The radial blocks of one row's descriptors into x: lanes over basis
// functions (two halves over neighbours), one shuffle between the halves.
// The Gaussian basis values use the hardware exponential (__expf: relative
// error within about 1e-6 for the arguments of the terms that matter, |x| < 10;
// the tiny far terms carry a few ulp more): the basis is the bulk of the
// radial work, and FP32 accuracy of the descriptors needs no more.
__device__ __forceinline__ void desc_radial(const NbStage &S, int n, const PotDev &P, int S_, float *x, int lane) {
    const int nr = P.n_rbf;
    float acc[kMaxSpecies];
#pragma unroll
    for (int s = 0; s < kMaxSpecies; ++s) acc[s] = 0.f;
    const int kb = lane & 15;
    if (kb < nr) {
        const float mu = (float)kb * P.rbf_w;
        for (int p = lane >> 4; p < n; p += 2) {
            const float t = S.r[p] - mu;
            const float v = __expf(-t * t * P.rbf_inv2w2) * S.c[p].x;
            const int sp = S.sp[p];
#pragma unroll
            for (int s = 0; s < kMaxSpecies; ++s) acc[s] += (sp == s) ? v : 0.f;
        }
    }
#pragma unroll
    for (int s = 0; s < kMaxSpecies; ++s) acc[s] += __shfl_down_sync(0xffffffffu, acc[s], 16);
    if (lane < nr)
        for (int s = 0; s < S_; ++s) x[s * nr + lane] = acc[s];
}

// The one-hot of the centre species si and the zero padding of a descriptor row.
__device__ __forceinline__ void desc_onehot(const PotDev &P, int S_, int si, float *x, int lane) {
    const int off = S_ * P.n_rbf + P.n_ang;
    for (int f = off + lane; f < P.d0p; f += 32) x[f] = (f == off + si) ? 1.f : 0.f;
}

// One row's descriptors into x [d0p]: the radial blocks, the 16 angular terms
// by lanes over the flattened neighbour pairs with one reduce-scatter, the
// one-hot of the centre species si and zero padding.  S_ species; the row's n
// neighbours are staged in S.
__device__ __forceinline__ void desc_row(const NbStage &S, int n, const PotDev &P, int S_, int si, float *x, int lane) {
    const int nr = P.n_rbf;
    desc_radial(S, n, P, S_, x, lane);
    // angular
    if (P.n_ang) {
        // per (zeta, eta) the pair (lambda = +1, lambda = -1) of sums of b^zeta E_eta fc_p fc_q, packed: one fused
        // multiply-add of a float pair per (zeta, eta); the prefactors 2^(1 - zeta) (powers of two) are applied
        // to the warp totals
        float2 acc[4][2];
#pragma unroll
        for (int z = 0; z < 4; ++z) acc[z][0] = acc[z][1] = make_float2(0.f, 0.f);
        const int npairs = n * (n - 1) / 2;
        PairIter it(n, lane);
        for (int t = lane; t < npairs; t += 32, it.next()) {
            const int p = it.p, q = it.q();
            const float4 gp = S.g[p], gq = S.g[q], cp = S.c[p], cq = S.c[q];
            const float c = (gp.x * gq.x + gp.y * gq.y + gp.z * gq.z) * (gp.w * gq.w);
            const float ff = cp.x * cq.x;
            const float E1 = cp.z * cq.z * ff, E2 = cp.w * cq.w * ff;
            const float2 e1 = make_float2(E1, E1), e2 = make_float2(E2, E2);
            const float2 b1 = make_float2(1.f + c, 1.f - c);
            const float2 b2 = __fmul2_rn(b1, b1), b4 = __fmul2_rn(b2, b2), b8 = __fmul2_rn(b4, b4);
            acc[0][0] = __ffma2_rn(b1, e1, acc[0][0]);
            acc[0][1] = __ffma2_rn(b1, e2, acc[0][1]);
            acc[1][0] = __ffma2_rn(b2, e1, acc[1][0]);
            acc[1][1] = __ffma2_rn(b2, e2, acc[1][1]);
            acc[2][0] = __ffma2_rn(b4, e1, acc[2][0]);
            acc[2][1] = __ffma2_rn(b4, e2, acc[2][1]);
            acc[3][0] = __ffma2_rn(b8, e1, acc[3][0]);
            acc[3][1] = __ffma2_rn(b8, e2, acc[3][1]);
        }
        // back to the feature order 4 z + 2 lambda + eta
        float a[kNAng];
#pragma unroll
        for (int z = 0; z < 4; ++z) {
            a[4 * z] = acc[z][0].x;
            a[4 * z + 1] = acc[z][1].x;
            a[4 * z + 2] = acc[z][0].y;
            a[4 * z + 3] = acc[z][1].y;
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
        // feature f = lane / 2 has zeta index f / 4: prefactor 2^(1 - zeta)
        const int zf = lane >> 3;
        const float pref = zf == 0 ? 1.f : (zf == 1 ? 0.5f : (zf == 2 ? 0.125f : 0.0078125f));
        if ((lane & 1) == 0) x[S_ * nr + (lane >> 1)] = a[0] * pref;
    }
    desc_onehot(P, S_, si, x, lane);
}

// The radial part of dE_i/dr_p: c = sum_k w_k g_k'(r_p), w = dE/dX of the
// radial block of neighbour p's species (the pair gradient is c d_p / r_p).
__device__ __forceinline__ float radial_dcoef(const NbStage &S, int p, const PotDev &P, const float *wbuf) {
    const int nr = P.n_rbf;
    const float rp = S.r[p], fp = S.c[p].x, dfp = S.c[p].y;
    float c = 0.f;
    const float *wr = wbuf + S.sp[p] * nr;
    for (int k = 0; k < nr; ++k) {
        const float t = rp - (float)k * P.rbf_w;
        const float phi = __expf(-t * t * P.rbf_inv2w2);
        c += wr[k] * phi * (-t * P.rbf_invw2 * fp + dfp);
    }
    return c;
}

// The pair gradients g_p = dE_i/d(r_p) of one row from its staged neighbours
// and its dE/dX (wbuf, shared memory): the angular pairs by diagonals d = 1 ..
// n/2 (pair (p, p + d mod n); for even n the last diagonal holds the n/2 pairs
// p < d), lane l owning neighbours p = l + 32 s (s < R, n <= 32 R); the p side
// of a pair stays in p's owner's registers, the q side is handed to q's owner
// through tb [n] in shared memory (within a diagonal the q are distinct).  Every
// neighbour's sums are formed in a fixed order (by diagonal), so the result does
// not depend on timing or launch shape.  Then per neighbour the radial term;
// g_p goes to pg[p], and its components are added to fx, fy, fz (lane-partial).
template <int R>
__device__ __forceinline__ void row_pair_grads(const NbStage &S, int n, const PotDev &P, int S_, const float *wbuf,
                                               float4 *tb, float4 *__restrict__ pg, int lane, float &fx, float &fy,
                                               float &fz) {
    const int nr = P.n_rbf;
    float wang[kNAng];   // dE/dX of the angular features
#pragma unroll
    for (int t = 0; t < kNAng; ++t) wang[t] = P.n_ang ? wbuf[S_ * nr + t] : 0.f;
    const AngW aw = ang_weights(wang);   // in registers across the pair loop
    float ax[R], ay[R], az[R], ab[R];
#pragma unroll
    for (int s = 0; s < R; ++s) ax[s] = ay[s] = az[s] = ab[s] = 0.f;
    if (P.n_ang) {
        for (int d = 1; 2 * d <= n; ++d) {
            const bool half = 2 * d == n;
#pragma unroll
            for (int s = 0; s < R; ++s) {
                const int p = lane + 32 * s;
                if (p < n && (!half || p < d)) {
                    const int q = p + d < n ? p + d : p + d - n;
                    tb[q] = pair_terms(S, aw, p, q, ax[s], ay[s], az[s], ab[s]);
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
#pragma unroll
    for (int s = 0; s < R; ++s) {
        const int p = lane + 32 * s;
        if (p >= n) continue;
        const float4 gp = S.g[p];
        const float xp = gp.x, yp = gp.y, zp = gp.z;
        const float rip = gp.w;
        const float c = radial_dcoef(S, p, P, wbuf);
        const float gx = c * xp * rip + ax[s] + ab[s] * xp;
        const float gy = c * yp * rip + ay[s] + ab[s] * yp;
        const float gz = c * zp * rip + az[s] + ab[s] * zp;
        pg[p] = make_float4(gx, gy, gz, 0.f);
        fx += gx;
        fy += gy;
        fz += gz;
    }
}

}  // namespace lsd
