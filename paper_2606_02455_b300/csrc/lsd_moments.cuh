// lsd_moments.cuh -- the sixteen angular features and their adjoint through
// Cartesian moments of the neighbour directions: the same functions as the
// pair sums of lsd_pairs.cuh, in O(n) work per row instead of O(n^2).
//
// With u_p = d_p / r_p, w_p^e = fc(r_p) exp(-eta_e r_p^2) and c_pq = u_p.u_q,
// every feature is a polynomial of degree zeta <= 8 in c summed over pairs:
//   T[z][l][e] = 2^(1-zeta) sum_{p<q} (1 + lambda c_pq)^zeta w_p^e w_q^e
//             = 2^(1-zeta) (1/2) [ sum_m C(zeta, m) lambda^m M_m^e - (1 + lambda)^zeta Q^e ],
// the sum over ordered pairs (p, q) less its diagonal c = 1, where
//   M_m^e = sum_{p,q} c_pq^m w_p^e w_q^e = sum_{|alpha| = m} (m! / alpha!) (Phi_alpha^e)^2,
//   Phi_alpha^e = sum_p w_p^e u_p^alpha,  Q^e = sum_p (w_p^e)^2
// (multinomial theorem, u^alpha = x^a y^b z^c; 165 monomials of degree <= 8).
//
// The adjoint: with W = dE/dT, gamma_m^e = dE/dM_m^e and kappa^e = dE/dQ^e are
// per-row scalars, Psi_alpha^e = dE/dPhi_alpha^e = 2 gamma_|alpha|^e (m!/alpha!)
// Phi_alpha^e, and for neighbour p, with F^e(u) = sum_alpha Psi_alpha^e u^alpha
// and G^e = grad F^e at u_p,
//   dE/dd_p = sum_e [ (F^e + 2 kappa^e w_p^e) w_p^e' u_p + (w_p^e / r_p) (G^e - (u_p.G^e) u_p) ]
// (w' = dw/dr; the bracket is the derivative of u_p with respect to d_p).  F
// and G come from one nested Horner evaluation over x, then y, then z.
//
// Monomials are indexed in the order c (outer), b, a (inner): the x-powers of
// one (b, c) column are consecutive.
#pragma once

#include "lsd_pairs.cuh"

namespace lsd {

constexpr int kMomDeg = 8;
constexpr int kMomAlpha = 165;              // (kMomDeg + 1)(kMomDeg + 2)(kMomDeg + 3) / 6
constexpr int kMomLd = 168;                 // one eta's moments, padded to a multiple of 4
constexpr int kMomFloats = 2 * kMomLd;      // one row: [eta][alpha]
constexpr int kMomRuns = 64;                // two runs of one or two monomials per lane
constexpr int kMomTab = 33;                 // floats per staged neighbour in the forward pass (odd: no bank conflicts)
// per warp: the powers [32][kMomTab], padding to 16 bytes, 32 float4 (x, w1, w2, species), 32 float2 (r, fc)
constexpr int kMomTabFloats = 32 * kMomTab + 4 + 128 + 64;

// index of the monomial (0, b, c), the first of its column: the planes c' < c
// (plane c' holds (D - c')(D - c' + 1) / 2 monomials, D = kMomDeg + 1), then
// the columns b' < b of plane c (column b' holds D - c - b')
__host__ __device__ constexpr int mom_col(int b, int c) {
    constexpr int D = kMomDeg + 1;
    return D * (D + 1) * (D + 2) / 6 - (D - c) * (D - c + 1) * (D - c + 2) / 6 + b * (D - c) - b * (b - 1) / 2;
}

__host__ __device__ constexpr float mom_fact(int m) {
    float f = 1.f;
    for (int i = 2; i <= m; ++i) f *= (float)i;
    return f;
}

// The forward pass accumulates only the moments of degree 8 and 7 (45 + 36 =
// 81 monomials): since |u| = 1, every lower degree follows exactly from the
// traces Phi_beta = Phi_{beta + 2 e_x} + Phi_{beta + 2 e_y} + Phi_{beta + 2 e_z}
// (u^beta (x^2 + y^2 + z^2) = u^beta), degree m - 2 from degree m.  Each lane
// owns two runs: a degree-7 monomial x^a y^b z^c with its degree-8 neighbour
// x^(a+1) y^b z^c (36 pairs), or a degree-8 monomial y^b z^(8-b) alone (9).  A
// run is (a, 9 + b, 18 + c) (offsets into a neighbour's staged powers) and its
// first index k0 and length.
struct MomRunTable {
    int4 run[kMomRuns];   // (a, 9 + b, 18 + c, k0 << 8 | len)
};
__host__ __device__ constexpr MomRunTable mom_run_table() {
    MomRunTable t{};
    int r = 0;
    for (int c = 0; c < kMomDeg; ++c)
        for (int b = 0; b < kMomDeg - c; ++b) {
            const int a = kMomDeg - 1 - b - c;
            t.run[r++] = int4{a, 9 + b, 18 + c, ((mom_col(b, c) + a) << 8) | 2};
        }
    for (int b = 0; b <= kMomDeg; ++b) t.run[r++] = int4{0, 9 + b, 18 + kMomDeg - b, (mom_col(b, kMomDeg - b) << 8) | 1};
    for (; r < kMomRuns; ++r) t.run[r] = int4{0, 9, 18, 0};   // empty run
    return t;
}
static_assert(mom_col(0, kMomDeg + 1) == kMomAlpha, "monomial count");

// (global memory, not constant: lanes read different entries, which the constant cache would serialise)
static __device__ const MomRunTable kMomRunTab = mom_run_table();

// The trace rounds: round q forms degrees 6 - 2q and 5 - 2q from degrees 8 - 2q
// and 7 - 2q; entry (dst, src1, src2, src3) of a degree-d monomial beta, the
// sources beta + 2 e_x, beta + 2 e_y, beta + 2 e_z.
constexpr int kMomTrace = kMomAlpha - 81;   // 84 monomials of degree <= 6
struct MomTraceTable {
    int4 e[kMomTrace];
    int start[5];   // round q: entries start[q] .. start[q + 1]
};
__host__ __device__ constexpr MomTraceTable mom_trace_table() {
    MomTraceTable t{};
    int i = 0, q = 0;
    for (int m = kMomDeg - 2; m >= 0; m -= 2, ++q) {
        t.start[q] = i;
        for (int d = m; d >= m - 1 && d >= 0; --d)
            for (int c = 0; c <= d; ++c)
                for (int b = 0; b <= d - c; ++b) {
                    const int a = d - b - c;
                    t.e[i++] = int4{mom_col(b, c) + a, mom_col(b, c) + a + 2, mom_col(b + 2, c) + a,
                                    mom_col(b, c + 2) + a};
                }
    }
    t.start[q] = i;
    return t;
}
static_assert(mom_trace_table().start[4] == kMomTrace, "trace entries");
static __device__ const MomTraceTable kMomTraceTab = mom_trace_table();

// Monomial indices by degree: degree m's (m + 1)(m + 2) / 2 indices from
// kMomDegStart[m] (the features need M_m = sum over one degree).
struct MomDegTable {
    int k[kMomAlpha];
};
__host__ __device__ constexpr MomDegTable mom_deg_table() {
    MomDegTable t{};
    int i = 0;
    for (int m = 0; m <= kMomDeg; ++m)
        for (int c = 0; c <= m; ++c)
            for (int b = 0; b <= m - c; ++b) t.k[i++] = mom_col(b, c) + m - b - c;
    return t;
}
static __device__ const MomDegTable kMomDegTab = mom_deg_table();
__host__ __device__ constexpr int mom_deg_start(int m) { return m * (m + 1) * (m + 2) / 6; }

// Per monomial: its degree and multinomial m! / alpha! (the adjoint's scaling).
struct MomCoefTable {
    float2 dm[kMomLd];
};
__host__ __device__ constexpr MomCoefTable mom_coef_table() {
    MomCoefTable t{};
    for (int c = 0; c <= kMomDeg; ++c)
        for (int b = 0; b <= kMomDeg - c; ++b)
            for (int a = 0; a <= kMomDeg - b - c; ++a)
                t.dm[mom_col(b, c) + a] = float2{(float)(a + b + c),
                                                 mom_fact(a + b + c) / (mom_fact(a) * mom_fact(b) * mom_fact(c))};
    return t;
}
static __device__ const MomCoefTable kMomCoefTab = mom_coef_table();

// C(zeta, m) lambda^m for zeta = 1, 2, 4, 8 ([z][m]) and lambda = +1; lambda = -1 flips odd m.
__host__ __device__ constexpr float mom_binom(int z, int m) {
    const int zeta = 1 << z;
    if (m > zeta) return 0.f;
    float v = 1.f;
    for (int i = 0; i < m; ++i) v = v * (float)(zeta - i) / (float)(i + 1);
    return v;
}

// One row's descriptors without a full staging of its neighbours: in chunks
// of 32, lane q forms neighbour q's geometry in registers (the operations of
// nb_stage_load) and stages its powers x^0..8, y^0..8, z^0..8 (rows of kMomTab
// floats: the odd length puts the 32 lanes' rows, and one row's entries, in
// distinct banks), (x, w1, w2, species) and (r, fc); then the radial blocks
// accumulate with lanes over basis functions (two halves over the chunk's
// neighbours, the order of desc_radial) and the top moments with lanes over
// runs.  x: the row's descriptors (radial blocks at 0, the sixteen angular
// features at S_ n_rbf); mom_out: the row's moments [e * kMomLd + k] (global);
// tab: this warp's kMomTabFloats floats, afterwards holding the moments.  The
// sums run over neighbours in list order and the traces in a fixed order: the
// result does not depend on the launch shape.
__device__ __forceinline__ void mom_row_descriptors(const uint4 *__restrict__ fj, uint4 fi,
                                                    const int *__restrict__ keys, int n, const Geo &g,
                                                    const PotDev &P, int S_, float *tab,
                                                    float *__restrict__ mom_out, float *x, int lane) {
    static_assert(32 * kMomTab >= kMomFloats, "the staging buffer holds the moments afterwards");
    float *phs = tab;
    float4 *xw = reinterpret_cast<float4 *>(tab + 32 * kMomTab + 4);
    float2 *rf = reinterpret_cast<float2 *>(tab + 32 * kMomTab + 4 + 128);
    const int4 r0 = kMomRunTab.run[lane], r1 = kMomRunTab.run[lane + 32];
    const int nr = P.n_rbf, kb = lane & 15, half = lane >> 4;
    const float mu = (float)kb * P.rbf_w;
    float racc[kMaxSpecies];
#pragma unroll
    for (int sp = 0; sp < kMaxSpecies; ++sp) racc[sp] = 0.f;
    float acc[2][2][2];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int s = 0; s < 2; ++s) acc[r][s][0] = acc[r][s][1] = 0.f;
    float q1 = 0.f, q2 = 0.f;
    for (int base = 0; base < n; base += 32) {
        const int p = base + lane;
        if (p < n) {
            const int key = keys[p];
            const uint4 fk = fj[key >> 5];
            const float3 d = entry_disp(fi, fk, key & 31, g);
            const float r2 = dist2_rule(d.x, d.y, d.z);
            const float r = sqrtf(r2);
            float fc, dfc;
            cutoff_fn(r, P.desc_rc, fc, dfc);
            const float ri = 1.f / r;
            const float e1 = expf(-0.005f * r2), e2 = expf(-0.05f * r2);
            const float ux = d.x * ri, uy = d.y * ri, uz = d.z * ri;
            const float w1 = fc * e1, w2 = fc * e2;
            q1 += w1 * w1;
            q2 += w2 * w2;
            float *t = tab + lane * kMomTab;
            float px = 1.f, py = 1.f, pz = 1.f;
#pragma unroll
            for (int k = 0; k <= kMomDeg; ++k) {
                t[k] = px;
                t[9 + k] = py;
                t[18 + k] = pz;
                px *= ux;
                py *= uy;
                pz *= uz;
            }
            xw[lane] = make_float4(ux, w1, w2, __int_as_float((int)fk.w));
            rf[lane] = make_float2(r, fc);
        }
        __syncwarp();
        const int cnt = n - base < 32 ? n - base : 32;
        if (kb < nr)
            for (int q = half; q < cnt; q += 2) {
                const float2 v = rf[q];
                const int sp = __float_as_int(xw[q].w);
                const float t = v.x - mu;
                const float b = __expf(-t * t * P.rbf_inv2w2) * v.y;
#pragma unroll
                for (int s2 = 0; s2 < kMaxSpecies; ++s2) racc[s2] += (sp == s2) ? b : 0.f;
            }
        for (int q = 0; q < cnt; ++q) {
            const float *t = tab + q * kMomTab;
            const float4 v = xw[q];
            const float vx = v.x, w1 = v.y, w2 = v.z;
            const float m0 = t[r0.x] * t[r0.y] * t[r0.z];
            const float m1 = t[r1.x] * t[r1.y] * t[r1.z];
            const float m0x = m0 * vx, m1x = m1 * vx;
            acc[0][0][0] = fmaf(w1, m0, acc[0][0][0]);
            acc[0][0][1] = fmaf(w2, m0, acc[0][0][1]);
            acc[0][1][0] = fmaf(w1, m0x, acc[0][1][0]);
            acc[0][1][1] = fmaf(w2, m0x, acc[0][1][1]);
            acc[1][0][0] = fmaf(w1, m1, acc[1][0][0]);
            acc[1][0][1] = fmaf(w2, m1, acc[1][0][1]);
            acc[1][1][0] = fmaf(w1, m1x, acc[1][1][0]);
            acc[1][1][1] = fmaf(w2, m1x, acc[1][1][1]);
        }
        __syncwarp();
    }
    // the radial blocks: the two halves' sums
#pragma unroll
    for (int sp = 0; sp < kMaxSpecies; ++sp) racc[sp] += __shfl_down_sync(0xffffffffu, racc[sp], 16);
    if (lane < nr) {
#pragma unroll
        for (int sp = 0; sp < kMaxSpecies; ++sp)
            if (sp < S_) x[sp * nr + lane] = racc[sp];
    }
    x += S_ * nr;   // the angular features follow
    // the top degrees into phs, then the lower degrees by traces
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int4 ru = r ? r1 : r0;
        const int k0 = ru.w >> 8, len = ru.w & 255;
#pragma unroll
        for (int s = 0; s < 2; ++s)
            if (s < len) {
                phs[k0 + s] = acc[r][s][0];
                phs[kMomLd + k0 + s] = acc[r][s][1];
            }
    }
    __syncwarp();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int e0 = kMomTraceTab.start[q], cntq = kMomTraceTab.start[q + 1] - e0;
        for (int t = lane; t < 2 * cntq; t += 32) {
            const int4 d = kMomTraceTab.e[e0 + (t >> 1)];
            float *ph = phs + (t & 1) * kMomLd;
            ph[d.x] = (ph[d.y] + ph[d.z]) + ph[d.w];
        }
        __syncwarp();
    }
    // moments out (coalesced), and the sums M_m^e degree by degree
    for (int k = lane; k < kMomLd; k += 32) {
        mom_out[k] = k < kMomAlpha ? phs[k] : 0.f;
        mom_out[kMomLd + k] = k < kMomAlpha ? phs[kMomLd + k] : 0.f;
    }
    float M0[kMomDeg + 1], M1[kMomDeg + 1];
#pragma unroll
    for (int m = 0; m <= kMomDeg; ++m) {
        float v0 = 0.f, v1 = 0.f;
        const int cm = (m + 1) * (m + 2) / 2;
#pragma unroll
        for (int j0 = 0; j0 < cm; j0 += 32)
            if (j0 + lane < cm) {
                const int k = kMomDegTab.k[mom_deg_start(m) + j0 + lane];
                const float mu = kMomCoefTab.dm[k].y, a0 = phs[k], a1 = phs[kMomLd + k];
                v0 = fmaf(mu * a0, a0, v0);
                v1 = fmaf(mu * a1, a1, v1);
            }
        M0[m] = warp_sum(v0);
        M1[m] = warp_sum(v1);
    }
    q1 = warp_sum(q1);
    q2 = warp_sum(q2);
    // feature f = 4 z + 2 l + e on lane f
    if (lane < kNAng) {
        const int z = lane >> 2, l = (lane >> 1) & 1, e = lane & 1;
        float acc_f = 0.f;
#pragma unroll
        for (int m = 0; m <= kMomDeg; ++m) {
            const float bz = z == 0 ? mom_binom(0, m) : (z == 1 ? mom_binom(1, m) : (z == 2 ? mom_binom(2, m) : mom_binom(3, m)));
            const float sg = (l && (m & 1)) ? -bz : bz;
            acc_f = fmaf(sg, e ? M1[m] : M0[m], acc_f);
        }
        const int zeta = 1 << z;
        const float diag = l ? 0.f : (float)(1 << zeta);   // (1 + lambda)^zeta
        const float pref = z == 0 ? 1.f : (z == 1 ? 0.5f : (z == 2 ? 0.125f : 0.0078125f));
        x[lane] = 0.5f * pref * (acc_f - diag * (e ? q2 : q1));
    }
}

// The adjoint scalars of one row, gk[e * 9 + m] = gamma_m^e = dE/dM_m^e and
// gk[18 + e] = kappa^e = dE/dQ^e, one per lane, from dE/dX of the sixteen
// angular features (wang, shared memory); gk is this warp's (shared memory).
__device__ __forceinline__ void mom_gamma_kappa(const float *wang, float *gk, int lane) {
    if (lane < 2 * (kMomDeg + 1) + 2) {
        float v = 0.f;
        if (lane < 2 * (kMomDeg + 1)) {
            const int e = lane / (kMomDeg + 1), m = lane % (kMomDeg + 1);
#pragma unroll
            for (int z = 0; z < 4; ++z) {
                const float pref = z == 0 ? 1.f : (z == 1 ? 0.5f : (z == 2 ? 0.125f : 0.0078125f));
                float bz = 0.f;
#pragma unroll
                for (int mm = 0; mm <= kMomDeg; ++mm)
                    if (mm == m) bz = mom_binom(z, mm);
                const float sg = (m & 1) ? -bz : bz;   // lambda = -1
                v += 0.5f * pref * (wang[4 * z + e] * bz + wang[4 * z + 2 + e] * sg);
            }
        } else {
            const int e = lane - 2 * (kMomDeg + 1);
#pragma unroll
            for (int z = 0; z < 4; ++z) {
                const float pref = z == 0 ? 1.f : (z == 1 ? 0.5f : (z == 2 ? 0.125f : 0.0078125f));
                v -= 0.5f * pref * wang[4 * z + e] * (float)(1 << (1 << z));   // lambda = +1: (1 + 1)^zeta
            }
        }
        gk[lane] = v;
    }
    __syncwarp();
}

// F^e(u) = sum_k Psi_k^e u^k and its gradient for both etas, by nested Horner
// schemes (x within a column, then y, then z); psi read by every lane at the
// same address (shared-memory broadcast).
__device__ __forceinline__ void mom_eval(const float2 *psi, float ux, float uy, float uz, float (&F)[2],
                                         float (&G)[2][3]) {
#pragma unroll
    for (int e = 0; e < 2; ++e) F[e] = G[e][0] = G[e][1] = G[e][2] = 0.f;
#pragma unroll
    for (int c = kMomDeg; c >= 0; --c) {
        // a compiler-only memory barrier: the coefficient loads of one z-power are scheduled within its block,
        // which bounds the registers the unrolled evaluation holds
        asm volatile("" ::: "memory");
        float H[2] = {0.f, 0.f}, Hx[2] = {0.f, 0.f}, Hy[2] = {0.f, 0.f};
#pragma unroll
        for (int b = kMomDeg - c; b >= 0; --b) {
            const int k0 = mom_col(b, c), L = kMomDeg + 1 - b - c;
            const float2 top = psi[k0 + L - 1];
            float h[2] = {top.x, top.y}, hd[2] = {0.f, 0.f};
#pragma unroll
            for (int a = L - 2; a >= 0; --a) {
                const float2 ps = psi[k0 + a];
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    hd[e] = (a == L - 2) ? h[e] : fmaf(hd[e], ux, h[e]);
                    h[e] = fmaf(h[e], ux, e ? ps.y : ps.x);
                }
            }
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                if (b == kMomDeg - c) {
                    H[e] = h[e];
                    Hx[e] = hd[e];
                } else {
                    Hy[e] = (b == kMomDeg - c - 1) ? H[e] : fmaf(Hy[e], uy, H[e]);
                    H[e] = fmaf(H[e], uy, h[e]);
                    Hx[e] = fmaf(Hx[e], uy, hd[e]);
                }
            }
        }
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            if (c == kMomDeg) {
                F[e] = H[e];
                G[e][0] = Hx[e];
                G[e][1] = Hy[e];
            } else {
                G[e][2] = (c == kMomDeg - 1) ? F[e] : fmaf(G[e][2], uz, F[e]);
                F[e] = fmaf(F[e], uz, H[e]);
                G[e][0] = fmaf(G[e][0], uz, Hx[e]);
                G[e][1] = fmaf(G[e][1], uz, Hy[e]);
            }
        }
    }
}

}  // namespace lsd
