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
constexpr int kMomRuns = 64;                // two runs of up to four monomials per lane
constexpr int kMomTab = 33;                 // floats per staged neighbour in the forward pass (odd: no bank conflicts)

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

// The forward pass: each lane owns two runs of up to four monomials
// x^a y^b z^c, a = a0 .. a0 + 3, of one column.  A run is (a0, 9 + b, 18 + c)
// (offsets into a neighbour's staged powers), its first index k0 and length,
// and the multinomials m! / alpha! of its four members.
struct MomRunTable {
    int4 run[kMomRuns];      // (a0, 9 + b, 18 + c, k0 << 8 | len)
    float4 mult[kMomRuns];
};
__host__ __device__ constexpr MomRunTable mom_run_table() {
    MomRunTable t{};
    int r = 0;
    for (int c = 0; c <= kMomDeg; ++c)
        for (int b = 0; b <= kMomDeg - c; ++b) {
            const int L = kMomDeg + 1 - b - c;
            for (int a0 = 0; a0 < L; a0 += 4) {
                const int len = L - a0 < 4 ? L - a0 : 4;
                t.run[r] = int4{a0, 9 + b, 18 + c, ((mom_col(b, c) + a0) << 8) | len};
                float m4[4] = {0.f, 0.f, 0.f, 0.f};
                for (int s = 0; s < len; ++s) {
                    const int a = a0 + s;
                    m4[s] = mom_fact(a + b + c) / (mom_fact(a) * mom_fact(b) * mom_fact(c));
                }
                t.mult[r] = float4{m4[0], m4[1], m4[2], m4[3]};
                ++r;
            }
        }
    for (; r < kMomRuns; ++r) {
        t.run[r] = int4{0, 9, 18, 0};   // empty run
        t.mult[r] = float4{0.f, 0.f, 0.f, 0.f};
    }
    return t;
}
static_assert(mom_col(0, kMomDeg + 1) == kMomAlpha, "monomial count");

// (global memory, not constant: lanes read different entries, which the constant cache would serialise)
static __device__ const MomRunTable kMomRunTab = mom_run_table();

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

// The angular features of one row (x[0 .. 15]) and its moments
// (mom_out[e * kMomLd + k], global) from the n staged neighbours of S.  tab:
// this warp's staging buffer of 32 neighbours x kMomTab floats (x^0..8,
// y^0..8, z^0..8 at 0, 9, 18; x, w1, w2 at 27, 28, 29; the odd row length
// puts the 32 lanes' rows, and one row's entries, in distinct banks).  The sums run over
// neighbours in list order for every lane: the result does not depend on the
// launch shape.
__device__ __forceinline__ void mom_forward(const NbStage &S, int n, float *tab, float *__restrict__ mom_out,
                                            float *x, int lane) {
    const int4 r0 = kMomRunTab.run[lane], r1 = kMomRunTab.run[lane + 32];
    float acc[2][4][2];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int s = 0; s < 4; ++s) acc[r][s][0] = acc[r][s][1] = 0.f;
    float q1 = 0.f, q2 = 0.f;
    for (int base = 0; base < n; base += 32) {
        const int p = base + lane;
        if (p < n) {
            const float4 gp = S.g[p], cp = S.c[p];
            const float ux = gp.x * gp.w, uy = gp.y * gp.w, uz = gp.z * gp.w;
            const float w1 = cp.x * cp.z, w2 = cp.x * cp.w;
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
            t[27] = ux;
            t[28] = w1;
            t[29] = w2;
        }
        __syncwarp();
        const int cnt = n - base < 32 ? n - base : 32;
        for (int q = 0; q < cnt; ++q) {
            const float *t = tab + q * kMomTab;
            const float vx = t[27], w1 = t[28], w2 = t[29];
            float m0 = t[r0.x] * t[r0.y] * t[r0.z];
            float m1 = t[r1.x] * t[r1.y] * t[r1.z];
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                acc[0][s][0] = fmaf(w1, m0, acc[0][s][0]);
                acc[0][s][1] = fmaf(w2, m0, acc[0][s][1]);
                acc[1][s][0] = fmaf(w1, m1, acc[1][s][0]);
                acc[1][s][1] = fmaf(w2, m1, acc[1][s][1]);
                m0 *= vx;
                m1 *= vx;
            }
        }
        __syncwarp();
    }
    // the moments out; each lane's contributions to M_m^e by degree
    float Mp[2][kMomDeg + 1];
#pragma unroll
    for (int m = 0; m <= kMomDeg; ++m) Mp[0][m] = Mp[1][m] = 0.f;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int4 ru = r ? r1 : r0;
        const float4 mu = r ? kMomRunTab.mult[lane + 32] : kMomRunTab.mult[lane];
        const int k0 = ru.w >> 8, len = ru.w & 255;
        const int d0 = ru.x + (ru.y - 9) + (ru.z - 18);   // degree of the run's first member
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            if (s < len) {
                mom_out[k0 + s] = acc[r][s][0];
                mom_out[kMomLd + k0 + s] = acc[r][s][1];
            }
            const float ms = s == 0 ? mu.x : (s == 1 ? mu.y : (s == 2 ? mu.z : mu.w));   // 0 past len
            const float v0 = ms * acc[r][s][0] * acc[r][s][0], v1 = ms * acc[r][s][1] * acc[r][s][1];
#pragma unroll
            for (int m = 0; m <= kMomDeg; ++m) {
                Mp[0][m] += (d0 + s == m) ? v0 : 0.f;
                Mp[1][m] += (d0 + s == m) ? v1 : 0.f;
            }
        }
    }
    if (lane < kMomLd - kMomAlpha) {
        mom_out[kMomAlpha + lane] = 0.f;
        mom_out[kMomLd + kMomAlpha + lane] = 0.f;
    }
#pragma unroll
    for (int m = 0; m <= kMomDeg; ++m) {
        Mp[0][m] = warp_sum(Mp[0][m]);
        Mp[1][m] = warp_sum(Mp[1][m]);
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
            acc_f = fmaf(sg, e ? Mp[1][m] : Mp[0][m], acc_f);
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
