// lsd_common.cuh -- device-side definitions shared by the kernels of liblsd.so.
//
// Counter-based noise (Philox4x32-10, Box-Muller), the fixed-point neighbour
// membership rule, and the parameter blocks passed to every kernel.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <stdint.h>

namespace lsd {

constexpr int kMaxSpecies = 4;
constexpr int kMaxLayers = 6;
constexpr int kMaxK = 128;
constexpr int kNAng = 16;

// ---------------------------------------------------------------------------
// Parameter blocks
// ---------------------------------------------------------------------------

struct Geo {
    int N;                 // atoms
    int S;                 // species
    double scale[3];       // 2^32 / L per axis (fixed-point wrap)
    float scale_f[3];      // fl32(L / 2^32) per axis
    float Lf[3];           // fl32(L) per axis
};

struct PotDev {
    int kind;              // LSD_POT_*
    int precision;         // LSD_FP32 | LSD_BF16 | LSD_FP8 | LSD_FP32_CUDA_CORES | LSD_FP32_TF32
    int head;              // LSD_HEAD_*
    float head_scale;
    int has_lj, has_mlp;
    float lj_rc2f;         // fl32(rc_lj^2)
    float desc_rc2f;       // fl32(rc_desc^2)
    float desc_rc;         // rc_desc
    float rmax2f;          // max of the two
    int n_rbf, n_ang, n_layers, width;
    int d0, d0p;           // input width and its padding to a multiple of 32
    float rbf_w, rbf_inv2w2, rbf_invw2;
    // LJ pair tables [si*S+sj]
    float lj_sig2[kMaxSpecies * kMaxSpecies];
    float lj_eps24[kMaxSpecies * kMaxSpecies];
    float lj_eps4[kMaxSpecies * kMaxSpecies];
    float lj_shift[kMaxSpecies * kMaxSpecies];
    // FP32 weights: Wt[l] = W_l^T padded [din_p][width]; Wn[l] = W_l padded [width][din_p]
    const float *Wt[kMaxLayers];
    const float *Wn[kMaxLayers];
    const float *b[kMaxLayers];
    const float *wout;
    float bout;
    // BF16 copies (same layouts)
    const __nv_bfloat16 *Wt_bf[kMaxLayers];
    const __nv_bfloat16 *Wn_bf[kMaxLayers];
    const __nv_bfloat16 *wout_bf;
};

struct Coef {
    double c1;             // exp(-gamma dt)
    double aF;             // (1 + c1) (dt/2) kappa
    double hm[kMaxSpecies];     // (dt/2) / m
    double sig[kMaxSpecies];    // sqrt(m kB T kappa (1 - exp(-2 gamma dt)))
    double aF_sig[kMaxSpecies]; // aF / sig
    uint64_t seed;
    // OBABO through the staggered frame (App. E)
    int obabo;                  // 0: ABOBA; 1: staggered OBABO (full-step A, no trailing A)
    double ch;                  // exp(-gamma dt / 2)
    double bF;                  // (dt/2) kappa: one B half-step per unit force
    double ob_a, ob_b;          // conditional law of the first half-step noise: mean ch / (1 + c1) w, sd sqrt(1/(1+c1))
    double hmf[kMaxSpecies];    // dt / m
    double sigh[kMaxSpecies];   // sqrt(m kB T kappa (1 - exp(-gamma dt)))
};

// Header of one window buffer of the pipelined loop: the step index of the
// state the window was drafted from, how many steps the draft reached, and
// whether the kernels that would (re)draft it skip.
struct WinHdr {
    long long base;
    int k_eff;
    int skip;
    int keep;   // the redraft's Verlet build: 1 when the speculative draft stands
};

// Device-resident run state.  step is the index of the base state.
struct DevState {
    long long step;
    long long target_step;       // windows stop committing at this step
    int n_commit_last;
    int first_reject_last;       // 1-based, -1 if none
    int k_eff;                   // window steps drafted (the draft stops early if an atom left the list's skin)
    int err;                     // bit flags: 1 neighbour overflow, 2 non-finite
    unsigned int blocks_done;    // last-block counter of the commit kernel
    unsigned grid_count, grid_gen;   // the transport's grid barrier: arrivals of this generation, generation
    long long windows, committed, rejected, verified;
    long long stages;                // verification passes (one per window, or one per stage run)
    // lists kept across windows (lsd_set_list_reuse): the draft stopped at the displacement bound (rebuild before
    // the next window), this window's verdict, and the number of list builds the verdicts asked for
    int list_force, list_rebuild, list_moved;
    unsigned list_done;   // blocks of the check kernel that finished (its last block resets it)
    long long list_builds;
    double sum_delta, sum_pred;
    // the pipelined loop's speculation policy (lsd_draft.cu; results do not depend on it): a running mean of
    // "the last committed window had no rejection", and whether the next round skips its speculative draft
    float spec_ema;
    int spec_hint;
    int accept[kMaxK];
    double logr[kMaxK], logu[kMaxK], dnorm[kMaxK];
};

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): 10 rounds of the 4x32 multiply-xor
// bijection; Weyl key schedule.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

__device__ __forceinline__ uint4 philox_words(uint64_t seed, uint64_t n, uint32_t atom, uint32_t stream) {
    return philox4x32_10(make_uint4((uint32_t)n, (uint32_t)(n >> 32), atom, stream),
                         make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
}

// Three standard normals for (step n, atom, stream): Box-Muller on 23-bit
// uniforms u1 = ((w0>>9)+1/2)/2^23, u2 = (w1>>9)/2^23; z from (w2, w3).
__device__ __forceinline__ float3 normals3(uint64_t seed, uint64_t n, uint32_t atom, uint32_t stream) {
    const uint4 w = philox_words(seed, n, atom, stream);
    const float u1 = ((float)(w.x >> 9) + 0.5f) * 0x1p-23f;
    const float u2 = (float)(w.y >> 9) * 0x1p-23f;
    const float u3 = ((float)(w.z >> 9) + 0.5f) * 0x1p-23f;
    const float u4 = (float)(w.w >> 9) * 0x1p-23f;
    const float r1 = sqrtf(-2.0f * logf(u1));
    const float r2 = sqrtf(-2.0f * logf(u3));
    float s1, c1, s2, c2;
    sincospif(2.0f * u2, &s1, &c1);
    sincospif(2.0f * u4, &s2, &c2);
    return make_float3(r1 * c1, r1 * s1, r2 * c2);
}

// Uniform in (0, 1] with 53 bits for the acceptance test of step n (stream 1).
__device__ __forceinline__ double uniform53(uint64_t seed, uint64_t n) {
    const uint4 w = philox_words(seed, n, 0u, 1u);
    const unsigned long long m = (unsigned long long)(w.x >> 5) * 67108864ull + (unsigned long long)(w.y >> 6) + 1ull;
    return (double)m * 0x1p-53;
}

// ---------------------------------------------------------------------------
// Fixed-point positions and the membership rule
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t fixpoint(double q, double scale) {
    // floor(fl64(q * scale)) as one round-toward-minus-infinity conversion
    const long long fi = __double2ll_rd(__dmul_rn(q, scale));
    return (uint32_t)(unsigned long long)fi;
}

// Entry s of a per-species array inside a by-value kernel parameter, by
// selection: a dynamic index would copy the whole parameter struct to local
// memory.
__device__ __forceinline__ double species_pick(const double (&a)[kMaxSpecies], int s) {
    return s == 0 ? a[0] : (s == 1 ? a[1] : (s == 2 ? a[2] : a[3]));
}

// Layer l's bias pointer by selection (a dynamic index into the by-value
// PotDev would copy it to local memory).
__device__ __forceinline__ const float *layer_bias(const PotDev &P, int l) {
    const float *b = P.b[0];
#pragma unroll
    for (int k = 1; k < kMaxLayers; ++k) b = l == k ? P.b[k] : b;
    return b;
}

// The OBABO output momentum of one coordinate of a staggered step (App. E):
// p_in = p_prev + (dt/2) kappa F; w = (p_new - c1 p_prev - (1 + c1)(dt/2) kappa F) / s_half;
// xi1 = ch/(1+c1) w + sqrt(1/(1+c1)) eta; p_mid = ch p_in + s_half xi1.
__device__ __forceinline__ double obabo_output(const Coef &cf, int sp, double pprev, double F, double pnew,
                                              double eta) {
    const double sh = species_pick(cf.sigh, sp);
    const double p_in = pprev + cf.bF * F;
    const double w = (pnew - cf.c1 * pprev - cf.aF * F) / sh;
    const double xi1 = cf.ob_a * w + cf.ob_b * eta;
    return cf.ch * p_in + sh * xi1;
}

__device__ __forceinline__ float dist2_rule(float dx, float dy, float dz) {
    return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}

__device__ __forceinline__ int shift_code(int sx, int sy, int sz) { return (sx + 1) + 3 * (sy + 1) + 9 * (sz + 1); }

__device__ __forceinline__ void code_shift(int code, int &sx, int &sy, int &sz) {
    sx = code % 3 - 1;
    sy = (code / 3) % 3 - 1;
    sz = code / 9 - 1;
}

// Along one axis: d0 = (int32)(u_j - u_i) is the minimum image in fixed point,
// k = (u_j - u_i - d0)/2^32 in {-1,0,1}; dmin = fl32(fl32(d0) * fl32(L/2^32));
// the image r in {-1,0,1} relative to it has displacement dmin (r = 0) or
// fl32(dmin + r fl32(L)), and absolute image shift s = r - k.  Only r = 0 and
// r = -sign(dmin) can lie within a cutoff rc < L.  Everything is 32-bit.
__device__ __forceinline__ void axis_min(uint32_t ui, uint32_t uj, float scale_f, float &dmin, int &k) {
    const int d0 = (int)(uj - ui);
    dmin = __fmul_rn(__int2float_rn(d0), scale_f);
    k = (uj >= ui) ? (d0 < 0 ? 1 : 0) : (d0 >= 0 ? -1 : 0);
}

// The (at most two) images of j along one axis that pass the per-axis bound
// d^2 < rc^2 (a necessary condition for membership), in ascending image order.
struct AxisOpts {
    float d0, d1;  // displacements
    int s0, s1;    // absolute image shifts
    int n;
};
__device__ __forceinline__ float opt_d(const AxisOpts &o, int b) { return b ? o.d1 : o.d0; }
__device__ __forceinline__ int opt_s(const AxisOpts &o, int b) { return b ? o.s1 : o.s0; }

__device__ __forceinline__ AxisOpts axis_opts(uint32_t ui, uint32_t uj, float scale_f, float Lf, float rc2f) {
    float dmin;
    int k;
    axis_min(ui, uj, scale_f, dmin, k);
    const int ra = dmin > 0.f ? -1 : 1;
    const float da = __fadd_rn(dmin, ra > 0 ? Lf : -Lf);
    const bool okm = __fmul_rn(dmin, dmin) < rc2f;
    const bool oka = (dmin != 0.f) && (__fmul_rn(da, da) < rc2f);
    AxisOpts o;
    o.d0 = o.d1 = 0.f;
    o.s0 = o.s1 = 0;
    o.n = 0;
    const float dfirst = ra < 0 ? da : dmin, dsecond = ra < 0 ? dmin : da;
    const int sfirst = ra < 0 ? ra - k : -k, ssecond = ra < 0 ? -k : ra - k;
    const bool okfirst = ra < 0 ? oka : okm, oksecond = ra < 0 ? okm : oka;
    if (okfirst) {
        o.d0 = dfirst;
        o.s0 = sfirst;
        o.n = 1;
        if (oksecond) {
            o.d1 = dsecond;
            o.s1 = ssecond;
            o.n = 2;
        }
    } else if (oksecond) {
        o.d0 = dsecond;
        o.s0 = ssecond;
        o.n = 1;
    }
    return o;
}

// Displacement of the stored neighbour entry (k, absolute shift code).
__device__ __forceinline__ float disp_from_shift(uint32_t ui, uint32_t uj, int s, float scale_f, float Lf) {
    float dmin;
    int k;
    axis_min(ui, uj, scale_f, dmin, k);
    const int r = s + k;
    return r == 0 ? dmin : __fadd_rn(dmin, r > 0 ? Lf : -Lf);
}

__device__ __forceinline__ float3 entry_disp(uint4 fi, uint4 fk, int code, const Geo &g) {
    int sx, sy, sz;
    code_shift(code, sx, sy, sz);
    return make_float3(disp_from_shift(fi.x, fk.x, sx, g.scale_f[0], g.Lf[0]),
                       disp_from_shift(fi.y, fk.y, sy, g.scale_f[1], g.Lf[1]),
                       disp_from_shift(fi.z, fk.z, sz, g.scale_f[2], g.Lf[2]));
}

// ---------------------------------------------------------------------------
// Small numeric helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ float sigmoidf_(float h) { return 1.0f / (1.0f + expf(-h)); }
__device__ __forceinline__ float siluf_(float h) { return h * sigmoidf_(h); }
__device__ __forceinline__ float dsiluf_(float h) {
    const float s = sigmoidf_(h);
    return s * (1.0f + h * (1.0f - s));
}
// SiLU and its derivative from one exponential and one reciprocal (hardware
// approximations, a few ulp): the tensor-core epilogues, where they are the
// bulk of the per-element work.  h is clamped at -80 so exp(-h) stays finite.
// rcp.approx: one special-function-unit operation, within 1 ulp (the
// correctly rounded reciprocal takes a refinement sequence on top)
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ void silu_dsilu_fast(float h, float &a, float &d) {
    const float e = __expf(-fmaxf(h, -80.f));
    const float s = rcp_approx(1.0f + e);
    a = h * s;
    d = s * (1.0f + h * (1.0f - s));
}
__device__ __forceinline__ float d2siluf_(float h) {
    const float s = sigmoidf_(h);
    return s * (1.0f - s) * (2.0f + h * (1.0f - 2.0f * s));
}

// Programmatic dependent launch: a kernel launched with launch_dependent() may
// start while the stream's previous kernel is still running; pdl_wait() blocks
// until that kernel (and so every earlier one) has finished and its writes are
// visible, and pdl_release() lets the stream's next kernel begin launching.
// Both are no-ops in a kernel launched the ordinary way.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// The pair-gradient slot of the reverse entry (k_p, i, -s_p) of neighbour p
// of row (j, i), found by binary search in k_p's sorted list; -1 (and error
// bit 4) when it is missing.
__device__ __forceinline__ int find_reverse(const int *__restrict__ near_keys, const int *__restrict__ n_near,
                                            int cap, int N, int j, int i, int p, int *err) {
    const int key = near_keys[((size_t)j * N + i) * cap + p];
    const int rk = j * N + (key >> 5);
    const int want = (i << 5) | (26 - (key & 31));
    const int *kk = near_keys + (size_t)rk * cap;
    int lo = 0, hi = n_near[rk] - 1;
    while (lo <= hi) {
        const int mid = (lo + hi) >> 1;
        const int v = kk[mid];
        if (v == want) return rk * cap + mid;
        if (v < want) lo = mid + 1;
        else hi = mid - 1;
    }
    atomicOr(err, 4);
    return -1;
}

// Cosine cutoff and its derivative.
__device__ __forceinline__ void cutoff_fn(float r, float rc, float &fc, float &dfc) {
    float s, c;
    sincospif(r / rc, &s, &c);
    fc = 0.5f * (c + 1.0f);
    dfc = -0.5f * 3.14159265358979f / rc * s;
}

// Angular term parameters: zeta in {1,2,4,8} (slowest), lambda in {+1,-1}, eta in {0.005, 0.05} (fastest).
__device__ __forceinline__ float ang_eta(int a) { return (a & 1) ? 0.05f : 0.005f; }
__device__ __forceinline__ float ang_lambda(int a) { return ((a >> 1) & 1) ? -1.0f : 1.0f; }
__device__ __forceinline__ int ang_zeta(int a) { return 1 << (a >> 2); }

}  // namespace lsd
