// lsd_plain.cu -- plain target-only ABOBA Langevin (Eq. 2), many steps in one
// launch: the baseline the speculative window is measured against, fused as
// tightly as the draft.
//
// For systems of up to kPlainMaxN atoms whose target network is FP32 (the
// LSD_FP32 family: the same FP32 function as the verification's, here on the
// CUDA cores).  One cooperative launch of G = N / A blocks of A warps spread
// over the SMs (A = 8 atoms per block, 4 when the shared memory of 8 does not
// fit); block b owns atoms [A b, A b + A), one warp per atom.  The network's
// weights stay in each block's shared memory for the whole launch.  Per step:
//   1. A: q_mid = q + (dt/2) p/m of the owned atoms (FP64), their fixed-point
//      positions to global memory; grid barrier.
//   2. every atom's position into shared memory; per owned atom: the LJ forces
//      over every candidate image within the cutoff (the membership rule of
//      the neighbour lists, gather form), the descriptor neighbour list
//      (sorted keys, also to global memory for the other blocks' reverse
//      look-ups), its staged geometry and the descriptors.
//   3. the per-atom MLP forward and input gradient of the owned rows, FP32 on
//      the CUDA cores: each thread one output column of the block's rows, the
//      resident weights read along rows (forward) or columns (backward) of one
//      padded W^T, activations as float4 broadcasts.
//   4. per owned atom: the pair gradients (row_pair_grads: radial and angular
//      terms in a fixed order), to global memory; grid barrier.
//   5. per owned atom: F_i = F_LJ + sum_p g_{i,p} - sum_p g_{k_p, rev(p)}, the
//      reverse entries found by binary search in k_p's sorted list; then B, O,
//      B, A in FP64 with the step's noise (Philox, keyed by the step index).
// The lists and pair gradients of step n are read in phase 5 and rewritten in
// phases 2 and 4 of step n + 1, after its first barrier, which no block passes
// before every block has finished phase 5 of step n; positions are rewritten
// in phase 1 of step n + 1, after the second barrier of step n, which follows
// every block's last read of them.  The grid barriers count arrivals on a
// counter cleared before each launch (every block resident: a cooperative
// launch) and give up after about two seconds: the block then records the
// timeout and stops, and the others give up at their next barrier.
#include "lsd_common.cuh"
#include "lsd_kernels.h"
#include "lsd_pairs.cuh"

#include <cmath>

namespace lsd {

constexpr int kPlainMaxWarps = 8;   // owned atoms per block (one warp each): 8, or 4 when 8 do not fit

// A barrier over the whole grid: thread 0 of each block arrives on the counter
// and waits for the end of its generation of `total` arrivals (acquire), giving
// up after 4e9 cycles (about two seconds at the maximum clock).
__device__ bool plain_grid_barrier(unsigned long long *ctr, unsigned total) {
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned long long arrive = atomicAdd(ctr, 1ull);
        const unsigned long long target = (arrive / total + 1ull) * total;
        int ok = 1;
        const long long t0 = clock64();
        for (;;) {
            unsigned long long v;
            asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(ctr) : "memory");
            if (v >= target) break;
            if (clock64() - t0 > 4000000000ll) {
                ok = 0;
                break;
            }
        }
        __threadfence();
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

// Shared-memory layout of one CTA (A owned rows, list capacity cap, N atoms).
struct PlainSmem {
    uint4 *fix;        // [N] positions of the step
    int *keys;         // [A][cap] descriptor neighbours of owned atoms (sorted)
    float *stage;      // [A][kNbStageFloats cap] staged geometry (NbStage per row)
    float4 *tb;        // [A][cap] pair hand-over
    float *x;          // [A][ld] descriptors, later dE/dX
    float *a0, *a1;    // [A][ld] activations / backward vectors
    float *spr;        // [L][A][W] SiLU'(h)
    float *dedy;       // [A]
    double *qmid;      // [A][3]
    float4 *fl;        // [A] LJ force + own pair-gradient sum
    int *cnt;          // [A] list lengths
    float *w;          // the network, resident for the whole launch: per layer W_l^T [din_p][W + 1]
                       // (one padding column: conflict-free both along rows and along columns),
                       // then b_l [W]; then w_out [W]
};

// Floats of the resident network (layers of W_l^T with a padding column, biases, output row).
__host__ __device__ inline size_t plain_weight_floats(int d0p, int W, int L) {
    size_t n = 0;
    for (int l = 0; l < L; ++l) n += (size_t)(l == 0 ? d0p : W) * (W + 1) + W;
    return n + W;
}

__host__ __device__ inline size_t plain_smem_layout(int N, int A, int cap, int d0p, int W, int L, PlainSmem *out,
                                                    char *base) {
    const int ld = d0p > W ? d0p : W;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o += (bytes + 15) & ~(size_t)15;
        return at;
    };
    const size_t o_fix = take((size_t)N * sizeof(uint4));
    const size_t o_keys = take((size_t)A * cap * sizeof(int));
    const size_t o_stage = take((size_t)A * kNbStageFloats * cap * sizeof(float));
    const size_t o_tb = take((size_t)A * cap * sizeof(float4));
    const size_t o_x = take((size_t)A * ld * sizeof(float));
    const size_t o_a0 = take((size_t)A * ld * sizeof(float));
    const size_t o_a1 = take((size_t)A * ld * sizeof(float));
    const size_t o_spr = take((size_t)L * A * W * sizeof(float));
    const size_t o_dedy = take((size_t)A * sizeof(float));
    const size_t o_qmid = take((size_t)A * 3 * sizeof(double));
    const size_t o_fl = take((size_t)A * sizeof(float4));
    const size_t o_cnt = take((size_t)A * sizeof(int));
    const size_t o_w = take(plain_weight_floats(d0p, W, L) * sizeof(float));
    if (out) {
        out->fix = (uint4 *)(base + o_fix);
        out->keys = (int *)(base + o_keys);
        out->stage = (float *)(base + o_stage);
        out->tb = (float4 *)(base + o_tb);
        out->x = (float *)(base + o_x);
        out->a0 = (float *)(base + o_a0);
        out->a1 = (float *)(base + o_a1);
        out->spr = (float *)(base + o_spr);
        out->dedy = (float *)(base + o_dedy);
        out->qmid = (double *)(base + o_qmid);
        out->fl = (float4 *)(base + o_fl);
        out->cnt = (int *)(base + o_cnt);
        out->w = (float *)(base + o_w);
    }
    return o;
}

// Layer weights by selection (a dynamic index into the by-value PotDev would
// copy it to local memory).
__device__ __forceinline__ const float *layer_wn(const PotDev &P, int l) {
    const float *w = P.Wn[0];
#pragma unroll
    for (int k = 1; k < kMaxLayers; ++k) w = l == k ? P.Wn[k] : w;
    return w;
}
__device__ __forceinline__ const float *layer_wt(const PotDev &P, int l) {
    const float *w = P.Wt[0];
#pragma unroll
    for (int k = 1; k < kMaxLayers; ++k) w = l == k ? P.Wt[k] : w;
    return w;
}

// out[r][c] = sum_k in[r][k] B(k, c) for rows r < A, columns c < ncol, with
// B(k, c) = Bs[k * ldb + c * cs] in shared memory (the resident W^T with
// ldb = W + 1, cs = 1 forward; W = its transpose, ldb = 1, cs = W + 1
// backward: lanes read consecutive or odd-strided words, conflict-free either
// way); thread t takes column c = t % ncol and rows t / ncol + RS j (RS =
// threads / ncol, at most four rows); in [A][ld] read as float4 broadcasts
// along k.  The sum runs over k in order.
__device__ __forceinline__ void plain_gemm(const float *__restrict__ in, int ld, int kd, const float *__restrict__ Bs,
                                           int ldb, int cs, int ncol, int A, float (&acc)[4], int &c, int &r0,
                                           int &rs) {
    const int t = threadIdx.x;
    const int nt = blockDim.x;
    rs = nt >= ncol ? nt / ncol : 1;
    c = t % ncol;
    r0 = t / ncol;
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[j] = 0.f;
    const float *bc = Bs + (size_t)c * cs;
    for (int k = 0; k < kd; k += 4) {
        const float w0 = bc[(size_t)(k + 0) * ldb], w1 = bc[(size_t)(k + 1) * ldb];
        const float w2 = bc[(size_t)(k + 2) * ldb], w3 = bc[(size_t)(k + 3) * ldb];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int r = r0 + rs * j;
            if (r < A) {
                const float4 a = *reinterpret_cast<const float4 *>(in + (size_t)r * ld + k);
                acc[j] = fmaf(a.x, w0, acc[j]);
                acc[j] = fmaf(a.y, w1, acc[j]);
                acc[j] = fmaf(a.z, w2, acc[j]);
                acc[j] = fmaf(a.w, w3, acc[j]);
            }
        }
    }
}

template <bool MINIMG, int R>
__global__ void __launch_bounds__(32 * kPlainMaxWarps)
    plain_fused_kernel(int n_steps, Geo g, PotDev P, Coef cf, const int *__restrict__ species, double *__restrict__ q,
                       double *__restrict__ p, uint4 *__restrict__ gfix, int *__restrict__ gkeys,
                       int *__restrict__ gcnt, float4 *__restrict__ gpg, int cap, unsigned long long *__restrict__ bar,
                       DevState *__restrict__ st) {
    extern __shared__ __align__(16) char smraw[];
    const int N = g.N;
    const int G = gridDim.x, cidx = blockIdx.x;
    const int A = blockDim.x >> 5;   // owned atoms
    const int nwarps = A, nthreads = blockDim.x;
    const int a0i = cidx * A, a1i = min(N, a0i + A);
    const int nown = a1i > a0i ? a1i - a0i : 0;
    const int W = P.width, L = P.n_layers, d0p = P.d0p;
    const int ld = d0p > W ? d0p : W;
    PlainSmem sm;
    plain_smem_layout(N, A, cap, d0p, W, L, &sm, smraw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long n0 = st->step, tgt = st->target_step;   // uniform: nothing writes them before the end
    const long long n_run = n0 >= tgt ? 0 : (tgt - n0 < n_steps ? tgt - n0 : n_steps);
    const float rmax2 = P.rmax2f;
    // the network into shared memory once per launch (it does not change between steps)
    if (P.has_mlp && n_run > 0) {
        float *w = sm.w;
        for (int l = 0; l < L; ++l) {
            const int dinp = l == 0 ? d0p : W;
            const float *src = layer_wt(P, l);   // [dinp][W]
            for (int e = tid; e < dinp * W; e += nthreads) {
                const int k = e / W, cc = e - k * W;
                w[(size_t)k * (W + 1) + cc] = __ldg(src + e);
            }
            w += (size_t)dinp * (W + 1);
            const float *bl = layer_bias(P, l);
            for (int e = tid; e < W; e += nthreads) w[e] = __ldg(bl + e);
            w += W;
        }
        for (int e = tid; e < W; e += nthreads) w[e] = __ldg(P.wout + e);
        __syncthreads();
    }
    // resident layer l: W_l^T at layer_ws[l], bias after it; w_out at the end
    auto layer_ws = [&](int l) {
        const float *w = sm.w;
        for (int m = 0; m < l; ++m) w += (size_t)(m == 0 ? d0p : W) * (W + 1) + W;
        return w;
    };
    const float *wout_s = sm.w + plain_weight_floats(d0p, W, L) - W;

    for (long long s = 0; s < n_run; ++s) {
        const unsigned long long n = (unsigned long long)(n0 + s + 1);
        // 1. A half-step of the owned atoms, fixed point out
        for (int ii = warp; ii < nown; ii += nwarps) {
            const int i = a0i + ii;
            const int sp = species[i];
            uint32_t u = 0;
            if (lane < 3) {
                const double qm = __dadd_rn(q[3 * i + lane], __dmul_rn(p[3 * i + lane], species_pick(cf.hm, sp)));
                sm.qmid[3 * ii + lane] = qm;
                u = fixpoint(qm, g.scale[lane]);
            }
            const uint32_t ux = __shfl_sync(0xffffffffu, u, 0), uy = __shfl_sync(0xffffffffu, u, 1),
                           uz = __shfl_sync(0xffffffffu, u, 2);
            if (lane == 0) gfix[i] = make_uint4(ux, uy, uz, (unsigned)sp);
        }
        if (!plain_grid_barrier(bar, (unsigned)G)) {
            if (tid == 0) atomicOr(&st->err, 16);
            return;
        }
        // 2. positions, LJ, lists, descriptors
        for (int k = tid; k < N; k += nthreads) sm.fix[k] = __ldcg(gfix + k);
        __syncthreads();
        for (int ii = warp; ii < nown; ii += nwarps) {
            const int i = a0i + ii;
            const uint4 fi = sm.fix[i];
            const int si = (int)fi.w;
            int *keys = sm.keys + (size_t)ii * cap;
            float fx = 0.f, fy = 0.f, fz = 0.f;
            int cnt = 0;
            for (int b0 = 0; b0 < N; b0 += 32) {
                const int k = b0 + lane;
                unsigned mn = 0u;                 // near images of this candidate, in enumeration (code) order
                unsigned long long codes = 0ull;  // their shift codes, 5 bits each
                int nim = 0;
                if (k < N) {
                    const uint4 fk = sm.fix[k];
                    const int pr = si * g.S + (int)fk.w;
                    const float sig2 = P.lj_sig2[pr], eps24 = P.lj_eps24[pr];
                    auto image = [&](float dx, float dy, float dz, int code) {
                        const float d2 = dist2_rule(dx, dy, dz);
                        if (P.has_lj && d2 < P.lj_rc2f) {
                            const float s2 = sig2 / d2;
                            const float s6 = s2 * s2 * s2, s12 = s6 * s6;
                            const float fr = -eps24 * (2.f * s12 - s6) / d2;
                            fx += fr * dx;
                            fy += fr * dy;
                            fz += fr * dz;
                        }
                        if (P.has_mlp && d2 < P.desc_rc2f) {
                            mn |= 1u << nim;
                            codes |= (unsigned long long)code << (5 * nim);
                        }
                        ++nim;
                    };
                    if (MINIMG) {
                        if (k != i) {
                            float dx, dy, dz;
                            int kx, ky, kz;
                            axis_min(fi.x, fk.x, g.scale_f[0], dx, kx);
                            axis_min(fi.y, fk.y, g.scale_f[1], dy, ky);
                            axis_min(fi.z, fk.z, g.scale_f[2], dz, kz);
                            image(dx, dy, dz, shift_code(-kx, -ky, -kz));
                        }
                    } else {
                        const AxisOpts ox = axis_opts(fi.x, fk.x, g.scale_f[0], g.Lf[0], rmax2);
                        const AxisOpts oy = axis_opts(fi.y, fk.y, g.scale_f[1], g.Lf[1], rmax2);
                        const AxisOpts oz = axis_opts(fi.z, fk.z, g.scale_f[2], g.Lf[2], rmax2);
                        for (int bz = 0; bz < oz.n; ++bz)
                            for (int by = 0; by < oy.n; ++by)
                                for (int bx = 0; bx < ox.n; ++bx) {
                                    if (k == i && opt_s(ox, bx) == 0 && opt_s(oy, by) == 0 && opt_s(oz, bz) == 0)
                                        continue;
                                    image(opt_d(ox, bx), opt_d(oy, by), opt_d(oz, bz),
                                          shift_code(opt_s(ox, bx), opt_s(oy, by), opt_s(oz, bz)));
                                }
                    }
                }
                // compaction in (candidate, code) order: the list comes out sorted by key
                const int nn = __popc(mn);
                int sc = nn;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int t = __shfl_up_sync(0xffffffffu, sc, o);
                    if (lane >= o) sc += t;
                }
                const int tot = __shfl_sync(0xffffffffu, sc, 31);
                int w = cnt + sc - nn;
                for (int c = 0; c < nim; ++c)
                    if (mn & (1u << c)) {
                        if (w < cap) keys[w] = (k << 5) | (int)((codes >> (5 * c)) & 31ull);
                        ++w;
                    }
                cnt += tot;
            }
            if (cnt > cap) {
                if (lane == 0) atomicOr(&st->err, 1);
                cnt = cap;
            }
            __syncwarp();
            fx = warp_sum(fx);
            fy = warp_sum(fy);
            fz = warp_sum(fz);
            if (lane == 0) {
                sm.fl[ii] = make_float4(fx, fy, fz, 0.f);
                sm.cnt[ii] = cnt;
                gcnt[i] = cnt;
            }
            for (int t = lane; t < cnt; t += 32) gkeys[(size_t)i * cap + t] = keys[t];
            if (P.has_mlp) {
                NbStage S = nb_stage_ptrs(sm.stage + (size_t)ii * kNbStageFloats * cap, cap);
                nb_stage_load(S, sm.fix, fi, keys, cnt, g, P.desc_rc, lane);
                desc_row(S, cnt, P, g.S, si, sm.x + (size_t)ii * ld, lane);
            }
        }
        __syncthreads();
        if (P.has_mlp) {
            // 3. MLP forward (SiLU' kept) and input gradient of the owned rows
            float acc[4];
            int c, r0, rs;
            const float *in = sm.x;
            float *out = sm.a0;
            int din = d0p;
            for (int l = 0; l < L; ++l) {
                const float *ws = layer_ws(l);
                plain_gemm(in, ld, din, ws, W + 1, 1, W, nown, acc, c, r0, rs);
                const float bias = ws[(size_t)din * (W + 1) + c];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int r = r0 + rs * j;
                    if (r < nown) {
                        const float h = acc[j] + bias;
                        out[(size_t)r * ld + c] = siluf_(h);
                        sm.spr[((size_t)l * A + r) * W + c] = dsiluf_(h);
                    }
                }
                __syncthreads();
                in = out;
                out = (out == sm.a0) ? sm.a1 : sm.a0;
                din = W;
            }
            // y = w_out . a_L + b_out and e'(y), one warp per row
            for (int r = warp; r < nown; r += nwarps) {
                float v = 0.f;
                for (int cc = lane; cc < W; cc += 32) v += in[(size_t)r * ld + cc] * wout_s[cc];
                v = warp_sum(v);
                if (lane == 0) {
                    const float y = v + P.bout;
                    float dedy;
                    if (P.head == 1) {
                        dedy = 1.f;
                    } else {
                        const float th = tanhf(y);
                        dedy = P.head_scale * (1.f - th * th);
                    }
                    sm.dedy[r] = dedy;
                }
            }
            __syncthreads();
            // g_L = e'(y) w_out * SiLU'(h_L)
            for (int e = tid; e < nown * W; e += nthreads) {
                const int r = e / W, cc = e - r * W;
                out[(size_t)r * ld + cc] = sm.dedy[r] * wout_s[cc] * sm.spr[((size_t)(L - 1) * A + r) * W + cc];
            }
            __syncthreads();
            in = out;
            out = (out == sm.a0) ? sm.a1 : sm.a0;
            for (int l = L - 1; l >= 0; --l) {
                const int dout = l == 0 ? d0p : W;
                plain_gemm(in, ld, W, layer_ws(l), 1, W + 1, dout, nown, acc, c, r0, rs);
                float *dst = l == 0 ? sm.x : out;   // dE/dX over the descriptors, no longer needed
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int r = r0 + rs * j;
                    if (r < nown)
                        dst[(size_t)r * ld + c] = l > 0 ? acc[j] * sm.spr[((size_t)(l - 1) * A + r) * W + c] : acc[j];
                }
                __syncthreads();
                in = out;
                out = (out == sm.a0) ? sm.a1 : sm.a0;
            }
            // 4. pair gradients of the owned rows
            for (int ii = warp; ii < nown; ii += nwarps) {
                const int i = a0i + ii;
                NbStage S = nb_stage_ptrs(sm.stage + (size_t)ii * kNbStageFloats * cap, cap);
                float fx = 0.f, fy = 0.f, fz = 0.f;
                row_pair_grads<R>(S, sm.cnt[ii], P, g.S, sm.x + (size_t)ii * ld, sm.tb + (size_t)ii * cap,
                                  gpg + (size_t)i * cap, lane, fx, fy, fz);
                fx = warp_sum(fx);
                fy = warp_sum(fy);
                fz = warp_sum(fz);
                if (lane == 0) {
                    float4 f = sm.fl[ii];
                    f.x += fx;
                    f.y += fy;
                    f.z += fz;
                    sm.fl[ii] = f;
                }
            }
        }
        if (!plain_grid_barrier(bar, (unsigned)G)) {
            if (tid == 0) atomicOr(&st->err, 16);
            return;
        }
        // 5. reverse pair gradients, then B O B A
        for (int ii = warp; ii < nown; ii += nwarps) {
            const int i = a0i + ii;
            float rx = 0.f, ry = 0.f, rz = 0.f;
            if (P.has_mlp) {
                const int *own = sm.keys + (size_t)ii * cap;
                for (int t = lane; t < sm.cnt[ii]; t += 32) {
                    // the entry (i, -shift) in neighbour k's sorted list, written by its CTA this step
                    const int key = own[t];
                    const int k = key >> 5;
                    const int want = (i << 5) | (26 - (key & 31));
                    const int *kk = gkeys + (size_t)k * cap;
                    int lo = 0, hi = __ldcg(gcnt + k) - 1, at = -1;
                    while (lo <= hi) {
                        const int mid = (lo + hi) >> 1;
                        const int v = __ldcg(kk + mid);
                        if (v == want) {
                            at = mid;
                            break;
                        }
                        if (v < want) lo = mid + 1;
                        else hi = mid - 1;
                    }
                    if (at < 0) {
                        atomicOr(&st->err, 4);
                        continue;
                    }
                    const float4 v = __ldcg(gpg + (size_t)k * cap + at);
                    rx += v.x;
                    ry += v.y;
                    rz += v.z;
                }
                rx = warp_sum(rx);
                ry = warp_sum(ry);
                rz = warp_sum(rz);
            }
            if (lane < 3) {
                const float4 f = sm.fl[ii];
                const float F = lane == 0 ? f.x - rx : (lane == 1 ? f.y - ry : f.z - rz);
                const int sp = species[i];
                const float3 xi = normals3(cf.seed, n, (uint32_t)i, 0u);
                const float xx = lane == 0 ? xi.x : (lane == 1 ? xi.y : xi.z);
                const int o = 3 * i + lane;
                const double mu = __dadd_rn(__dmul_rn(cf.c1, p[o]), __dmul_rn(cf.aF, (double)F));
                const double pn = __dadd_rn(mu, __dmul_rn(species_pick(cf.sig, sp), (double)xx));
                p[o] = pn;
                q[o] = __dadd_rn(sm.qmid[3 * ii + lane], __dmul_rn(pn, species_pick(cf.hm, sp)));
            }
        }
        // the next step's phase 1 reads only this CTA's own atoms (written above by the same warp)
    }
    if (cidx == 0 && tid == 0 && n_run > 0) st->step = n0 + n_run;
}

static const void *plain_kernel_ptr(bool minimg, int R) {
    switch (R) {
        case 1: return minimg ? (const void *)plain_fused_kernel<true, 1> : (const void *)plain_fused_kernel<false, 1>;
        case 2: return minimg ? (const void *)plain_fused_kernel<true, 2> : (const void *)plain_fused_kernel<false, 2>;
        case 3: return minimg ? (const void *)plain_fused_kernel<true, 3> : (const void *)plain_fused_kernel<false, 3>;
        default: return minimg ? (const void *)plain_fused_kernel<true, 4> : (const void *)plain_fused_kernel<false, 4>;
    }
}

PlainPlan plain_plan(int N, const PotDev &P, bool fp32_target, bool obabo, int cap, const Geo &g, size_t max_smem) {
    PlainPlan pl{};
    pl.ok = false;
    if (N < 1 || N > kPlainMaxN || obabo) return pl;
    if (P.has_mlp) {
        if (!fp32_target || P.n_layers < 1 || P.n_layers > 4) return pl;
        if (!(P.width == 32 || P.width == 64 || P.width == 128)) return pl;
        if (!(P.d0p == 32 || P.d0p == 64 || P.d0p == 128)) return pl;
        if (P.n_rbf > 16 || (P.n_ang != 0 && P.n_ang != kNAng)) return pl;
    }
    if (cap > 128 || cap % 32) return pl;
    int A = kPlainMaxWarps;
    size_t smem = 0;
    for (; A >= 4; A /= 2) {
        smem = plain_smem_layout(N, A, cap, P.d0p, P.width, P.n_layers > 0 ? P.n_layers : 1, nullptr, nullptr);
        if (smem <= max_smem) break;
    }
    if (A < 4) return pl;
    const float lmin = fminf(g.Lf[0], fminf(g.Lf[1], g.Lf[2]));
    pl.minimg = std::sqrt((double)P.rmax2f) < 0.499 * (double)lmin;
    pl.atoms = A;
    pl.blocks = (N + A - 1) / A;
    pl.smem = smem;
    pl.cap = cap;
    pl.R = cap / 32;
    pl.ok = true;
    return pl;
}

cudaError_t plain_setup(const PlainPlan &pl) {
    const void *k = plain_kernel_ptr(pl.minimg, pl.R);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem);
    if (e != cudaSuccess) return e;
    // every block must be resident at once (the grid barriers wait for all of them)
    int dev = 0, sms = 0, per_sm = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 32 * pl.atoms, pl.smem);
    if (e != cudaSuccess) return e;
    return sms * per_sm >= pl.blocks ? cudaSuccess : cudaErrorCooperativeLaunchTooLarge;
}

template <bool MINIMG, int R>
static cudaError_t launch_plain_t(const PlainPlan &pl, int n_steps, const Geo &g, const PotDev &P, const Coef &cf,
                                  const int *species, double *q, double *p, uint4 *gfix, int *gkeys, int *gcnt,
                                  float4 *gpg, unsigned long long *bar, DevState *st, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(pl.blocks, 1, 1);
    cfg.blockDim = dim3(32 * pl.atoms, 1, 1);
    cfg.dynamicSmemBytes = pl.smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, plain_fused_kernel<MINIMG, R>, n_steps, g, P, cf, species, q, p, gfix, gkeys, gcnt,
                              gpg, pl.cap, bar, st);
}

cudaError_t launch_plain_fused(const PlainPlan &pl, int n_steps, const Geo &g, const PotDev &P, const Coef &cf,
                               const int *species, double *q, double *p, uint4 *gfix, int *gkeys, int *gcnt,
                               float4 *gpg, unsigned long long *bar, DevState *st, cudaStream_t s) {
    // the barrier counter starts each launch at zero (stream-ordered after the previous launch)
    cudaError_t e = cudaMemsetAsync(bar, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    switch (pl.R) {
        case 1: return pl.minimg ? launch_plain_t<true, 1>(pl, n_steps, g, P, cf, species, q, p, gfix, gkeys, gcnt, gpg, bar, st, s)
                                 : launch_plain_t<false, 1>(pl, n_steps, g, P, cf, species, q, p, gfix, gkeys, gcnt, gpg, bar, st, s);
        case 2: return pl.minimg ? launch_plain_t<true, 2>(pl, n_steps, g, P, cf, species, q, p, gfix, gkeys, gcnt, gpg, bar, st, s)
                                 : launch_plain_t<false, 2>(pl, n_steps, g, P, cf, species, q, p, gfix, gkeys, gcnt, gpg, bar, st, s);
        case 3: return pl.minimg ? launch_plain_t<true, 3>(pl, n_steps, g, P, cf, species, q, p, gfix, gkeys, gcnt, gpg, bar, st, s)
                                 : launch_plain_t<false, 3>(pl, n_steps, g, P, cf, species, q, p, gfix, gkeys, gcnt, gpg, bar, st, s);
        default: return pl.minimg ? launch_plain_t<true, 4>(pl, n_steps, g, P, cf, species, q, p, gfix, gkeys, gcnt, gpg, bar, st, s)
                                  : launch_plain_t<false, 4>(pl, n_steps, g, P, cf, species, q, p, gfix, gkeys, gcnt, gpg, bar, st, s);
    }
}

}  // namespace lsd
