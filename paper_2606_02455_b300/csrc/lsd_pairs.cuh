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

// One row's descriptors into x [d0p]: radial blocks by lanes over basis
// functions (two halves over neighbours), the 16 angular terms by lanes over
// the flattened neighbour pairs with one reduce-scatter, the one-hot of the
// centre species si and zero padding.  S_ species; the row's n neighbours are
// staged in S.
__device__ __forceinline__ void desc_row(const NbStage &S, int n, const PotDev &P, int S_, int si, float *x, int lane) {
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
            for (int s = 0; s < S_; ++s) x[s * nr + lane] = acc[s];
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
        if ((lane & 1) == 0) x[S_ * nr + (lane >> 1)] = a[0];
    }
    // one-hot and padding
    const int off = S_ * nr + P.n_ang;
    for (int f = off + lane; f < P.d0p; f += 32) x[f] = (f == off + si) ? 1.f : 0.f;
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
    float wang[kNAng];   // dE/dX of the angular features, in registers across the pair loop
#pragma unroll
    for (int t = 0; t < kNAng; ++t) wang[t] = P.n_ang ? wbuf[S_ * nr + t] : 0.f;
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
#pragma unroll
    for (int s = 0; s < R; ++s) {
        const int p = lane + 32 * s;
        if (p >= n) continue;
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
