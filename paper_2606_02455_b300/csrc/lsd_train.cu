// lsd_train.cu -- learned draft: target-labelled frames and force matching.
//
// Frames: every verified window step j contributes (q_mid_j, F_target_j) to a
// device ring buffer; committed and flushed steps alike, since each is an
// exact target label at a configuration the dynamics visits.
//
// Force matching of the draft E~ = LJ + sum_i y(x_i; theta), y an MLP with
// one hidden layer and a linear output: loss L = mean_{frames, components}
// |F~ - F*|^2.  With r = F~ - F* and the descriptor JVP v_i = (dx_i/dq) r,
// dL/dtheta = -(2/(F*3N)) sum_i d/dtheta [ v_i . dy/dx (x_i) ], which for
// h = W1 x + b1, t = W1 v is
//   d/dw_out[u] = t_u SiLU'(h_u)
//   d/db1[u]    = w_out[u] t_u SiLU''(h_u)
//   d/dW1[u][f] = w_out[u] (v_f SiLU'(h_u) + t_u SiLU''(h_u) x_f)
// (the double backward through MLP and descriptors, written out).  One CTA per
// frame computes the draft forces, the residual, the JVP and the per-weight
// sums over atoms in a fixed order; a second kernel sums frames in a fixed
// order and applies Adam.  Everything is FP32 (the BF16 copies are only for
// inference in the draft kernel).
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "lsd.h"
#include "lsd_common.cuh"
#include "lsd_train.h"

namespace lsd {

constexpr int kTrainThreads = 256;
constexpr int kTrainWarps = kTrainThreads / 32;
constexpr int kTrainCap = 96;
constexpr int kTrainMaxN = 256;

struct TrainGeo {
    int N, S, d0, W, n_rbf;
    float desc_rc, desc_rc2f, lj_rc2f, rc2_all;
    float rbf_w, rbf_inv2w2, rbf_invw2;
    int has_lj;
};

__device__ __forceinline__ void stage_members(const TrainGeo &T, const Geo &g, const uint4 *sfix, int i, float *sr,
                                              float *sa, int *ssp, const float4 *res, int &n_out) {
    // members of atom i within the descriptor cutoff, with r and (for the JVP) d-hat . (r_k - r_i)
    const int lane = threadIdx.x & 31;
    const uint4 fi = sfix[i];
    int cnt = 0;
    for (int base = 0; base < T.N; base += 32) {
        const int k = base + lane;
        unsigned m = 0u;
        AxisOpts ox, oy, oz;
        ox = oy = oz = AxisOpts{0.f, 0.f, 0, 0, 0};
        if (k < T.N) {
            const uint4 fk = sfix[k];
            ox = axis_opts(fi.x, fk.x, g.scale_f[0], g.Lf[0], T.desc_rc2f);
            oy = axis_opts(fi.y, fk.y, g.scale_f[1], g.Lf[1], T.desc_rc2f);
            oz = axis_opts(fi.z, fk.z, g.scale_f[2], g.Lf[2], T.desc_rc2f);
            for (int bz = 0; bz < oz.n; ++bz)
                for (int by = 0; by < oy.n; ++by)
                    for (int bx = 0; bx < ox.n; ++bx) {
                        if (k == i && opt_s(ox, bx) == 0 && opt_s(oy, by) == 0 && opt_s(oz, bz) == 0) continue;
                        if (dist2_rule(opt_d(ox, bx), opt_d(oy, by), opt_d(oz, bz)) < T.desc_rc2f) m |= 1u << (bx + 2 * by + 4 * bz);
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
            if (w < kTrainCap) {
                const float dx = opt_d(ox, c & 1), dy = opt_d(oy, (c >> 1) & 1), dz = opt_d(oz, c >> 2);
                const float r = sqrtf(dist2_rule(dx, dy, dz));
                sr[w] = r;
                ssp[w] = (int)sfix[k].w;
                if (res) {
                    const float4 rk = res[k], ri = res[i];
                    sa[w] = (dx * (rk.x - ri.x) + dy * (rk.y - ri.y) + dz * (rk.z - ri.z)) / r;
                }
            }
            ++w;
        }
        cnt += tot;
    }
    __syncwarp();
    n_out = cnt < kTrainCap ? cnt : kTrainCap;
}

__global__ void __launch_bounds__(kTrainThreads)
    fm_frame_kernel(TrainGeo T, Geo g, PotDev P, const float *__restrict__ w, const int *__restrict__ species,
                    const double *__restrict__ fq, const float *__restrict__ fF, long long frame0, long long n_avail,
                    float scale, float *__restrict__ grad_frames, float *__restrict__ loss_frames) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int N = T.N, d0 = T.d0, W = T.W;
    uint4 *sfix = (uint4 *)smraw;
    float4 *sres = (float4 *)(sfix + N);
    float *sx = (float *)(sres + N);       // [N][d0]
    float *sg = sx + (size_t)N * d0;       // [N][d0] dE/dx
    float *sv = sg + (size_t)N * d0;       // [N][d0] JVP
    float *sh = sv + (size_t)N * d0;       // [N][W]
    float *stt = sh + (size_t)N * W;       // [N][W] t = W1 v
    float *stage = stt + (size_t)N * W;    // per warp 3*kTrainCap
    float *sloss = stage + (size_t)kTrainWarps * 3 * kTrainCap;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long frame = (frame0 + blockIdx.x) % n_avail;
    const double *q = fq + (size_t)frame * 3 * N;
    const float *Fs = fF + (size_t)frame * 3 * N;
    const float *W1 = w, *b1 = w + (size_t)W * d0, *wo = b1 + W;
    float *my = stage + (size_t)warp * 3 * kTrainCap;
    float *sr = my, *sa = my + kTrainCap;
    int *ssp = (int *)(my + 2 * kTrainCap);
    for (int i = tid; i < N; i += blockDim.x)
        sfix[i] = make_uint4(fixpoint(q[3 * i], g.scale[0]), fixpoint(q[3 * i + 1], g.scale[1]),
                             fixpoint(q[3 * i + 2], g.scale[2]), (unsigned)species[i]);
    __syncthreads();
    // A: descriptors, hidden pre-activations, dE/dx
    for (int i = warp; i < N; i += kTrainWarps) {
        int n;
        stage_members(T, g, sfix, i, sr, sa, ssp, nullptr, n);
        float acc[kMaxSpecies];
#pragma unroll
        for (int s = 0; s < kMaxSpecies; ++s) acc[s] = 0.f;
        const int kb = lane & 15;
        if (kb < T.n_rbf) {
            const float mu = (float)kb * T.rbf_w;
            for (int p = lane >> 4; p < n; p += 2) {
                float fc, dfc;
                cutoff_fn(sr[p], T.desc_rc, fc, dfc);
                const float t = sr[p] - mu;
                const float v = expf(-t * t * T.rbf_inv2w2) * fc;
#pragma unroll
                for (int s = 0; s < kMaxSpecies; ++s) acc[s] += (ssp[p] == s) ? v : 0.f;
            }
        }
#pragma unroll
        for (int s = 0; s < kMaxSpecies; ++s) acc[s] += __shfl_down_sync(0xffffffffu, acc[s], 16);
        float *x = sx + (size_t)i * d0;
        for (int f = lane; f < d0; f += 32) x[f] = 0.f;
        __syncwarp();
        if (lane < T.n_rbf)
            for (int s = 0; s < T.S; ++s) x[s * T.n_rbf + lane] = acc[s];
        if (lane == 0) x[T.S * T.n_rbf + (int)sfix[i].w] = 1.f;
        __syncwarp();
        float gu = 0.f;
        if (lane < W) {
            float h = b1[lane];
            for (int f = 0; f < d0; ++f) h = fmaf(W1[(size_t)lane * d0 + f], x[f], h);
            sh[(size_t)i * W + lane] = h;
            gu = wo[lane] * dsiluf_(h);
        }
        for (int f = 0; f < d0; ++f) {
            const float vv = warp_sum(lane < W ? W1[(size_t)lane * d0 + f] * gu : 0.f);
            if (lane == 0) sg[(size_t)i * d0 + f] = vv;
        }
        __syncwarp();
    }
    __syncthreads();
    // B: draft forces and residual
    float lossw = 0.f;
    for (int i = warp; i < N; i += kTrainWarps) {
        const uint4 fi = sfix[i];
        const int si = (int)fi.w;
        float fx = 0.f, fy = 0.f, fz = 0.f;
        for (int k = lane; k < N; k += 32) {
            const uint4 fk = sfix[k];
            const AxisOpts ox = axis_opts(fi.x, fk.x, g.scale_f[0], g.Lf[0], T.rc2_all);
            if (!ox.n) continue;
            const AxisOpts oy = axis_opts(fi.y, fk.y, g.scale_f[1], g.Lf[1], T.rc2_all);
            if (!oy.n) continue;
            const AxisOpts oz = axis_opts(fi.z, fk.z, g.scale_f[2], g.Lf[2], T.rc2_all);
            const int pr = si * g.S + (int)fk.w;
            for (int bz = 0; bz < oz.n; ++bz)
                for (int by = 0; by < oy.n; ++by)
                    for (int bx = 0; bx < ox.n; ++bx) {
                        if (k == i && opt_s(ox, bx) == 0 && opt_s(oy, by) == 0 && opt_s(oz, bz) == 0) continue;
                        const float dx = opt_d(ox, bx), dy = opt_d(oy, by), dz = opt_d(oz, bz);
                        const float d2 = dist2_rule(dx, dy, dz);
                        if (T.has_lj && d2 < T.lj_rc2f) {
                            const float s2 = P.lj_sig2[pr] / d2;
                            const float s6 = s2 * s2 * s2, s12 = s6 * s6;
                            const float fr = -P.lj_eps24[pr] * (2.f * s12 - s6) / d2;
                            fx += fr * dx;
                            fy += fr * dy;
                            fz += fr * dz;
                        }
                        if (d2 < T.desc_rc2f) {
                            const float r = sqrtf(d2);
                            float fc, dfc;
                            cutoff_fn(r, T.desc_rc, fc, dfc);
                            const float *gi = sg + (size_t)i * d0 + (int)fk.w * T.n_rbf;
                            const float *gk = sg + (size_t)k * d0 + si * T.n_rbf;
                            float c = 0.f;
                            for (int b = 0; b < T.n_rbf; ++b) {
                                const float t = r - (float)b * T.rbf_w;
                                c += (gi[b] + gk[b]) * expf(-t * t * T.rbf_inv2w2) * (-t * T.rbf_invw2 * fc + dfc);
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
        if (lane == 0) {
            const float rx = fx - Fs[3 * i], ry = fy - Fs[3 * i + 1], rz = fz - Fs[3 * i + 2];
            sres[i] = make_float4(rx, ry, rz, 0.f);
            lossw += rx * rx + ry * ry + rz * rz;
        }
    }
    if (lane == 0) sloss[warp] = lossw;
    __syncthreads();
    // C: JVP v_i and t_i = W1 v_i
    for (int i = warp; i < N; i += kTrainWarps) {
        int n;
        stage_members(T, g, sfix, i, sr, sa, ssp, sres, n);
        float acc[kMaxSpecies];
#pragma unroll
        for (int s = 0; s < kMaxSpecies; ++s) acc[s] = 0.f;
        const int kb = lane & 15;
        if (kb < T.n_rbf) {
            const float mu = (float)kb * T.rbf_w;
            for (int p = lane >> 4; p < n; p += 2) {
                float fc, dfc;
                cutoff_fn(sr[p], T.desc_rc, fc, dfc);
                const float t = sr[p] - mu;
                const float dg = expf(-t * t * T.rbf_inv2w2) * (-t * T.rbf_invw2 * fc + dfc);
#pragma unroll
                for (int s = 0; s < kMaxSpecies; ++s) acc[s] += (ssp[p] == s) ? dg * sa[p] : 0.f;
            }
        }
#pragma unroll
        for (int s = 0; s < kMaxSpecies; ++s) acc[s] += __shfl_down_sync(0xffffffffu, acc[s], 16);
        float *v = sv + (size_t)i * d0;
        for (int f = lane; f < d0; f += 32) v[f] = 0.f;
        __syncwarp();
        if (lane < T.n_rbf)
            for (int s = 0; s < T.S; ++s) v[s * T.n_rbf + lane] = acc[s];
        __syncwarp();
        if (lane < W) {
            float t = 0.f;
            for (int f = 0; f < d0; ++f) t = fmaf(W1[(size_t)lane * d0 + f], v[f], t);
            stt[(size_t)i * W + lane] = t;
        }
        __syncwarp();
    }
    __syncthreads();
    // D: per-weight sums over atoms in order
    const int nw = W * d0 + 2 * W + 1;
    float *gout = grad_frames + (size_t)blockIdx.x * nw;
    for (int e = tid; e < nw; e += blockDim.x) {
        float acc = 0.f;
        if (e < W * d0) {
            const int u = e / d0, f = e - u * d0;
            for (int i = 0; i < N; ++i) {
                const float h = sh[(size_t)i * W + u];
                acc += wo[u] * (sv[(size_t)i * d0 + f] * dsiluf_(h) + stt[(size_t)i * W + u] * d2siluf_(h) *
                                                                          sx[(size_t)i * d0 + f]);
            }
        } else if (e < W * d0 + W) {
            const int u = e - W * d0;
            for (int i = 0; i < N; ++i) acc += wo[u] * stt[(size_t)i * W + u] * d2siluf_(sh[(size_t)i * W + u]);
        } else if (e < W * d0 + 2 * W) {
            const int u = e - W * d0 - W;
            for (int i = 0; i < N; ++i) acc += stt[(size_t)i * W + u] * dsiluf_(sh[(size_t)i * W + u]);
        }
        gout[e] = scale * acc;
    }
    if (tid == 0) {
        float l = 0.f;
        for (int k = 0; k < kTrainWarps; ++k) l += sloss[k];
        loss_frames[blockIdx.x] = -0.5f * scale * l;   // scale = -2/(F*3N)
    }
}

__global__ void fm_reduce_kernel(const float *__restrict__ grad_frames, const float *__restrict__ loss_frames,
                                 int n_frames, int nw, float *__restrict__ grad, float *__restrict__ loss) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < nw) {
        float s = 0.f;
        for (int f = 0; f < n_frames; ++f) s += grad_frames[(size_t)f * nw + e];
        grad[e] = s;
    }
    if (e == 0) {
        float l = 0.f;
        for (int f = 0; f < n_frames; ++f) l += loss_frames[f];
        *loss = l;
    }
}

__global__ void adam_kernel(float *__restrict__ w, float *__restrict__ m, float *__restrict__ v,
                            const float *__restrict__ grad, int nw, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nw) return;
    const float gr = grad[e];
    const float mm = b1 * m[e] + (1.f - b1) * gr;
    const float vv = b2 * v[e] + (1.f - b2) * gr * gr;
    m[e] = mm;
    v[e] = vv;
    w[e] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
}

__global__ void frame_capture_kernel(const double *__restrict__ w_qmid, const float *__restrict__ w_Ft, int K, int N,
                                     long long cap, long long start_verified, const DevState *__restrict__ st,
                                     const int *__restrict__ keff, double *__restrict__ fq, float *__restrict__ fF,
                                     int j0) {
    if (st->step >= st->target_step) return;
    const int j = j0 + blockIdx.y;   // window steps j0 .. K - 1 (a window verified in stages: one stage's)
    if (j >= *keff) return;   // steps the draft did not reach carry no target label
    // frames are numbered by verified window steps (the commit kernel adds k_eff afterwards)
    const long long slot = (st->verified - start_verified + j) % cap;
    const int D = 3 * N;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < D; e += gridDim.x * blockDim.x) {
        fq[slot * D + e] = w_qmid[(size_t)j * D + e];
        fF[slot * D + e] = w_Ft[(size_t)j * D + e];
    }
}

// ---------------------------------------------------------------------------
static TrainGeo make_tgeo(const TrainState &t, const PotDev &P) {
    TrainGeo T{};
    T.N = t.N;
    T.S = t.S;
    T.d0 = t.d0;
    T.W = t.W;
    T.n_rbf = P.n_rbf;
    T.desc_rc = P.desc_rc;
    T.desc_rc2f = P.desc_rc2f;
    T.lj_rc2f = P.lj_rc2f;
    T.rc2_all = fmaxf(P.lj_rc2f, P.desc_rc2f);
    T.rbf_w = P.rbf_w;
    T.rbf_inv2w2 = P.rbf_inv2w2;
    T.rbf_invw2 = P.rbf_invw2;
    T.has_lj = P.has_lj;
    return T;
}

static size_t fm_smem(const TrainState &t) {
    return (size_t)t.N * (sizeof(uint4) + sizeof(float4)) +
           ((size_t)t.N * (3 * t.d0 + 2 * t.W) + (size_t)kTrainWarps * 3 * kTrainCap + kTrainWarps) * sizeof(float);
}

int train_init(TrainState &t, const PotDev &P, const std::vector<float> &weights, int N) {
    t.enabled = P.kind == LSD_POT_LEARNED && P.has_mlp;
    if (!t.enabled) return LSD_OK;
    t.N = N;
    t.S = (P.d0 - P.n_ang) / (P.n_rbf + 1);
    t.d0 = P.d0;
    t.W = P.width;
    t.n_rbf = P.n_rbf;
    t.n_weights = weights.size();
    if (cudaMalloc(&t.w, t.n_weights * sizeof(float)) != cudaSuccess) return LSD_ENOMEM;
    if (cudaMalloc(&t.m, t.n_weights * sizeof(float)) != cudaSuccess) return LSD_ENOMEM;
    if (cudaMalloc(&t.v, t.n_weights * sizeof(float)) != cudaSuccess) return LSD_ENOMEM;
    if (cudaMalloc(&t.grad, t.n_weights * sizeof(float)) != cudaSuccess) return LSD_ENOMEM;
    if (cudaMalloc(&t.loss, sizeof(float)) != cudaSuccess) return LSD_ENOMEM;
    cudaMemset(t.m, 0, t.n_weights * sizeof(float));
    cudaMemset(t.v, 0, t.n_weights * sizeof(float));
    if (cudaMemcpy(t.w, weights.data(), t.n_weights * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
        return LSD_ECUDA;
    if (N <= kTrainMaxN &&
        cudaFuncSetAttribute(fm_frame_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024) != cudaSuccess)
        return LSD_ECUDA;
    return LSD_OK;
}

void train_free(TrainState &t) {
    for (void *p : {(void *)t.w, (void *)t.m, (void *)t.v, (void *)t.grad, (void *)t.loss, (void *)t.fq, (void *)t.fF,
                    (void *)t.grad_frames, (void *)t.loss_frames, (void *)t.lH, (void *)t.lT, (void *)t.lV,
                    (void *)t.lres, (void *)t.lFd, (void *)t.lloss, (void *)t.lpart})
        if (p) cudaFree(p);
    t = TrainState{};
}

int train_set_weights(TrainState &t, const std::vector<float> &w) {
    if (!t.enabled) return LSD_OK;
    if (w.size() != t.n_weights) return LSD_EINVAL;
    if (cudaMemcpy(t.w, w.data(), w.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) return LSD_ECUDA;
    return LSD_OK;
}

int train_get_weights(TrainState &t, std::vector<float> &w, cudaStream_t s) {
    if (!t.enabled) return LSD_EINVAL;
    w.resize(t.n_weights);
    if (cudaMemcpyAsync(w.data(), t.w, t.n_weights * sizeof(float), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return LSD_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return LSD_ECUDA;
    return LSD_OK;
}

int train_set_capture(TrainState &t, long long capacity, int N) {
    if (t.fq) cudaFree(t.fq);
    if (t.fF) cudaFree(t.fF);
    t.fq = nullptr;
    t.fF = nullptr;
    t.capture_on = capacity > 0;
    t.capacity = capacity;
    t.N = N;
    if (!t.capture_on) return LSD_OK;
    if (cudaMalloc(&t.fq, (size_t)capacity * 3 * N * sizeof(double)) != cudaSuccess) return LSD_ENOMEM;
    if (cudaMalloc(&t.fF, (size_t)capacity * 3 * N * sizeof(float)) != cudaSuccess) return LSD_ENOMEM;
    // frames are counted from the current verified-steps counter
    if (t.st) {
        DevState s;
        if (cudaMemcpy(&s, t.st, sizeof(DevState), cudaMemcpyDeviceToHost) != cudaSuccess) return LSD_ECUDA;
        t.start_verified = s.verified;
    }
    return LSD_OK;
}

int train_frame_count(TrainState &t, int64_t *n, cudaStream_t s) {
    *n = 0;
    if (!t.capture_on || !t.st) return LSD_OK;
    DevState ds;
    if (cudaMemcpyAsync(&ds, t.st, sizeof(DevState), cudaMemcpyDeviceToHost, s) != cudaSuccess) return LSD_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return LSD_ECUDA;
    const long long f = ds.verified - t.start_verified;
    *n = f < t.capacity ? f : t.capacity;
    return LSD_OK;
}

// Host copies of frames first .. first+count-1 (numbered from the start of
// capture); only the last `capacity` frames are still in the ring.
int train_get_frames(TrainState &t, long long first, long long count, double *q, float *F, cudaStream_t s) {
    if (!t.capture_on || !t.st) return LSD_ESTATE;
    DevState ds;
    if (cudaMemcpyAsync(&ds, t.st, sizeof(DevState), cudaMemcpyDeviceToHost, s) != cudaSuccess) return LSD_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return LSD_ECUDA;
    const long long total = ds.verified - t.start_verified;
    const long long oldest = total > t.capacity ? total - t.capacity : 0;
    if (first < oldest || first + count > total) return LSD_EINVAL;
    const size_t D = (size_t)3 * t.N;
    for (long long f = first; f < first + count; ++f) {
        const size_t slot = (size_t)(f % t.capacity), r = (size_t)(f - first);
        if (q && cudaMemcpyAsync(q + r * D, t.fq + slot * D, D * sizeof(double), cudaMemcpyDeviceToHost, s) !=
                     cudaSuccess)
            return LSD_ECUDA;
        if (F && cudaMemcpyAsync(F + r * D, t.fF + slot * D, D * sizeof(float), cudaMemcpyDeviceToHost, s) !=
                     cudaSuccess)
            return LSD_ECUDA;
    }
    return cudaStreamSynchronize(s) == cudaSuccess ? LSD_OK : LSD_ECUDA;
}

void enqueue_frame_capture(TrainState &t, const double *w_qmid, const float *w_Ft, int K, int N, DevState *st,
                           const int *keff, cudaStream_t s, int j0) {
    t.st = st;
    const int D = 3 * N;
    const int bx = (D + 255) / 256 < 64 ? (D + 255) / 256 : 64;
    frame_capture_kernel<<<dim3(bx, K - j0), 256, 0, s>>>(w_qmid, w_Ft, K, N, t.capacity, t.start_verified, st, keff,
                                                          t.fq, t.fF, j0);
}

// ---------------------------------------------------------------------------
// Frames larger than one block's shared memory: the same gradient with the
// frame's atoms as rows of the library's batched kernels (neighbour lists,
// descriptors, pair gradients and the force gather, run by the caller with
// the draft's parameters) and four kernels of its own:
//   fm_mlp_kernel       h = W1 x + b1 and dE/dx = W1^T (w_out SiLU'(h)) per row
//                       (FP32 master weights; the draft forces then come from
//                       the pair-gradient and gather kernels);
//   fm_residual_kernel  r_i = F~_i - F*_i and |r_i|^2 per row;
//   fm_jvp_kernel       v_i = sum_p phi_k'(r_ip) dhat_ip . (r_{k_p} - r_i) per
//                       species block, and t_i = W1 v_i;
//   fm_wgrad_kernel     the per-weight sums of the double backward over rows,
//                       per block of rows in order, then the blocks in order.
// Deterministic: no atomics, fixed summation orders.
// ---------------------------------------------------------------------------
constexpr int kFmRowsPerBlock = 256;

static int ensure_frame_bufs(TrainState &t, int n_frames);

__global__ void fm_mlp_kernel(int M, int d0, int d0p, int W, const float *__restrict__ w, const float *__restrict__ X,
                              float *__restrict__ H, float *__restrict__ G) {
    const int row = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= M) return;
    const float *W1 = w, *b1 = w + (size_t)W * d0, *wo = b1 + W;
    const float x = lane < d0 ? X[(size_t)row * d0p + lane] : 0.f;
    float h = 0.f, gu = 0.f;
    if (lane < W) h = b1[lane];
    for (int f = 0; f < d0; ++f) {
        const float xf = __shfl_sync(0xffffffffu, x, f);
        if (lane < W) h = fmaf(W1[(size_t)lane * d0 + f], xf, h);
    }
    if (lane < W) {
        H[(size_t)row * W + lane] = h;
        gu = wo[lane] * dsiluf_(h);   // linear head: dE/dy = 1
    }
    float g = 0.f;
    for (int u = 0; u < W; ++u) {
        const float gv = __shfl_sync(0xffffffffu, gu, u);
        if (lane < d0) g = fmaf(W1[(size_t)u * d0 + lane], gv, g);
    }
    if (lane < d0p) G[(size_t)row * d0p + lane] = g;
}

__global__ void fm_residual_kernel(int M, const float *__restrict__ Fd, const float *__restrict__ Fs,
                                   float4 *__restrict__ res, float *__restrict__ loss_rows) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    const float rx = Fd[3 * (size_t)i] - Fs[3 * (size_t)i], ry = Fd[3 * (size_t)i + 1] - Fs[3 * (size_t)i + 1],
                rz = Fd[3 * (size_t)i + 2] - Fs[3 * (size_t)i + 2];
    res[i] = make_float4(rx, ry, rz, 0.f);
    loss_rows[i] = rx * rx + ry * ry + rz * rz;
}

__global__ void fm_jvp_kernel(int M, int d0, int d0p, int W, const float *__restrict__ w, const uint4 *__restrict__ fix,
                              const int *__restrict__ near_keys, const int *__restrict__ n_near, int cap, Geo g,
                              PotDev P, const float4 *__restrict__ res, float *__restrict__ V,
                              float *__restrict__ T) {
    extern __shared__ __align__(16) float fsm[];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row = blockIdx.x * (blockDim.x >> 5) + wib;
    if (row >= M) return;
    float *sr = fsm + (size_t)wib * (3 * cap + 32), *sa = sr + cap;
    int *ssp = (int *)(sa + cap);
    float *sv = (float *)(ssp + cap);   // [32] v of this row
    const uint4 fi = fix[row];
    const float4 ri = res[row];
    const int n = min(n_near[row], cap);
    const int *keys = near_keys + (size_t)row * cap;
    for (int p = lane; p < n; p += 32) {
        const int key = keys[p];
        const int k = key >> 5;
        const uint4 fk = fix[k];
        const float3 d = entry_disp(fi, fk, key & 31, g);
        const float r = sqrtf(dist2_rule(d.x, d.y, d.z));
        const float4 rk = res[k];
        sr[p] = r;
        sa[p] = (d.x * (rk.x - ri.x) + d.y * (rk.y - ri.y) + d.z * (rk.z - ri.z)) / r;
        ssp[p] = (int)fk.w;
    }
    __syncwarp();
    float acc[kMaxSpecies];
#pragma unroll
    for (int s = 0; s < kMaxSpecies; ++s) acc[s] = 0.f;
    const int kb = lane & 15;
    if (kb < P.n_rbf) {
        const float mu = (float)kb * P.rbf_w;
        for (int p = lane >> 4; p < n; p += 2) {
            float fc, dfc;
            cutoff_fn(sr[p], P.desc_rc, fc, dfc);
            const float t = sr[p] - mu;
            const float dg = expf(-t * t * P.rbf_inv2w2) * (-t * P.rbf_invw2 * fc + dfc);
#pragma unroll
            for (int s = 0; s < kMaxSpecies; ++s) acc[s] += (ssp[p] == s) ? dg * sa[p] : 0.f;
        }
    }
#pragma unroll
    for (int s = 0; s < kMaxSpecies; ++s) acc[s] += __shfl_down_sync(0xffffffffu, acc[s], 16);
    sv[lane] = 0.f;
    __syncwarp();
    if (lane < P.n_rbf)
        for (int s = 0; s < g.S; ++s) sv[s * P.n_rbf + lane] = acc[s];
    __syncwarp();
    if (lane < d0p) V[(size_t)row * d0p + lane] = lane < d0 ? sv[lane] : 0.f;
    if (lane < W) {
        float t = 0.f;
        for (int f = 0; f < d0; ++f) t = fmaf(w[(size_t)lane * d0 + f], sv[f], t);
        T[(size_t)row * W + lane] = t;
    }
}

// Per block of kFmRowsPerBlock rows, every weight's sum over the rows in order;
// partials [blocks][nw].
__global__ void fm_wgrad_kernel(int M, int d0, int d0p, int W, const float *__restrict__ w,
                                const float *__restrict__ X, const float *__restrict__ H, const float *__restrict__ V,
                                const float *__restrict__ T, float *__restrict__ partials) {
    const int nw = W * d0 + 2 * W + 1;
    const float *wo = w + (size_t)W * d0 + W;
    const int r0 = blockIdx.x * kFmRowsPerBlock, r1 = min(M, r0 + kFmRowsPerBlock);
    for (int e = threadIdx.x; e < nw; e += blockDim.x) {
        float acc = 0.f;
        if (e < W * d0) {
            const int u = e / d0, f = e - u * d0;
            for (int i = r0; i < r1; ++i) {
                const float h = H[(size_t)i * W + u];
                acc += wo[u] * (V[(size_t)i * d0p + f] * dsiluf_(h) + T[(size_t)i * W + u] * d2siluf_(h) *
                                                                          X[(size_t)i * d0p + f]);
            }
        } else if (e < W * d0 + W) {
            const int u = e - W * d0;
            for (int i = r0; i < r1; ++i) acc += wo[u] * T[(size_t)i * W + u] * d2siluf_(H[(size_t)i * W + u]);
        } else if (e < W * d0 + 2 * W) {
            const int u = e - W * d0 - W;
            for (int i = r0; i < r1; ++i) acc += T[(size_t)i * W + u] * dsiluf_(H[(size_t)i * W + u]);
        }
        partials[(size_t)blockIdx.x * nw + e] = acc;
    }
}

// One frame's gradient and loss from the row-block partials, in block order.
__global__ void fm_frame_sum_kernel(const float *__restrict__ partials, int n_blocks, int nw,
                                    const float *__restrict__ loss_rows, int M, float scale,
                                    float *__restrict__ grad_frame, float *__restrict__ loss_frame) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < nw) {
        float s = 0.f;
        for (int b = 0; b < n_blocks; ++b) s += partials[(size_t)b * nw + e];
        grad_frame[e] = scale * s;
    }
    if (e == 0) {
        float l = 0.f;
        for (int i = 0; i < M; ++i) l += loss_rows[i];
        *loss_frame = -0.5f * scale * l;   // scale = -2/(F*3N)
    }
}

bool train_frame_fits(const TrainState &t) { return t.N <= kTrainMaxN; }

int train_large_bufs(TrainState &t, int n_frames) {
    const int M = t.N, d0p = (t.d0 + 31) / 32 * 32;
    if (!t.lH) {
        const size_t nb = (size_t)(M + kFmRowsPerBlock - 1) / kFmRowsPerBlock;
        if (cudaMalloc(&t.lH, (size_t)M * t.W * sizeof(float)) != cudaSuccess ||
            cudaMalloc(&t.lT, (size_t)M * t.W * sizeof(float)) != cudaSuccess ||
            cudaMalloc(&t.lV, (size_t)M * d0p * sizeof(float)) != cudaSuccess ||
            cudaMalloc(&t.lres, (size_t)M * sizeof(float4)) != cudaSuccess ||
            cudaMalloc(&t.lFd, (size_t)M * 3 * sizeof(float)) != cudaSuccess ||
            cudaMalloc(&t.lloss, (size_t)M * sizeof(float)) != cudaSuccess ||
            cudaMalloc(&t.lpart, nb * t.n_weights * sizeof(float)) != cudaSuccess)
            return LSD_ENOMEM;
    }
    return ensure_frame_bufs(t, n_frames);
}

void launch_fm_mlp(const TrainState &t, const float *X, int d0p, float *G, cudaStream_t s) {
    const int M = t.N;
    fm_mlp_kernel<<<(M * 32 + 255) / 256, 256, 0, s>>>(M, t.d0, d0p, t.W, t.w, X, t.lH, G);
}

void launch_fm_frame_grad(const TrainState &t, const uint4 *fix, const int *near_keys, const int *n_near, int cap,
                          const Geo &g, const PotDev &P, const float *X, int d0p, const float *Fstar, float scale,
                          int frame_index, cudaStream_t s) {
    const int M = t.N;
    fm_residual_kernel<<<(M + 255) / 256, 256, 0, s>>>(M, t.lFd, Fstar, t.lres, t.lloss);
    const int warps = 8;
    const size_t sm = (size_t)warps * (3 * cap + 32) * sizeof(float);
    fm_jvp_kernel<<<(M + warps - 1) / warps, warps * 32, sm, s>>>(M, t.d0, d0p, t.W, t.w, fix, near_keys, n_near, cap, g,
                                                                  P, t.lres, t.lV, t.lT);
    const int nb = (M + kFmRowsPerBlock - 1) / kFmRowsPerBlock;
    fm_wgrad_kernel<<<nb, 256, 0, s>>>(M, t.d0, d0p, t.W, t.w, X, t.lH, t.lV, t.lT, t.lpart);
    const int nw = (int)t.n_weights;
    fm_frame_sum_kernel<<<(nw + 255) / 256, 256, 0, s>>>(t.lpart, nb, nw, t.lloss, M, scale,
                                                         t.grad_frames + (size_t)frame_index * nw,
                                                         t.loss_frames + frame_index);
}

void launch_fm_reduce_adam(TrainState &t, int n_frames, bool adam, float lr, cudaStream_t s) {
    const int nw = (int)t.n_weights;
    fm_reduce_kernel<<<(nw + 255) / 256, 256, 0, s>>>(t.grad_frames, t.loss_frames, n_frames, nw, t.grad, t.loss);
    if (!adam) return;
    ++t.adam_t;
    ++t.iter;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)t.adam_t), c2 = 1.f - powf(b2, (float)t.adam_t);
    adam_kernel<<<(nw + 255) / 256, 256, 0, s>>>(t.w, t.m, t.v, t.grad, nw, lr, b1, b2, 1e-8f, c1, c2);
}

size_t train_adam_size(const TrainState &t) { return t.enabled ? t.n_weights : 0; }

int train_adam_get(TrainState &t, float *m, float *v) {
    if (!t.enabled) return LSD_OK;
    if (cudaMemcpy(m, t.m, t.n_weights * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess) return LSD_ECUDA;
    if (cudaMemcpy(v, t.v, t.n_weights * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess) return LSD_ECUDA;
    return LSD_OK;
}

int train_adam_set(TrainState &t, const float *m, const float *v) {
    if (!t.enabled) return LSD_OK;
    if (cudaMemcpy(t.m, m, t.n_weights * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) return LSD_ECUDA;
    if (cudaMemcpy(t.v, v, t.n_weights * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) return LSD_ECUDA;
    return LSD_OK;
}

static int ensure_frame_bufs(TrainState &t, int n_frames) {
    if (n_frames <= t.max_frames) return LSD_OK;
    if (t.grad_frames) cudaFree(t.grad_frames);
    if (t.loss_frames) cudaFree(t.loss_frames);
    t.grad_frames = nullptr;
    t.loss_frames = nullptr;
    if (cudaMalloc(&t.grad_frames, (size_t)n_frames * t.n_weights * sizeof(float)) != cudaSuccess) return LSD_ENOMEM;
    if (cudaMalloc(&t.loss_frames, (size_t)n_frames * sizeof(float)) != cudaSuccess) return LSD_ENOMEM;
    t.max_frames = n_frames;
    return LSD_OK;
}

static int fm_launch(TrainState &t, const Geo &g, const PotDev &P, const int *species, const double *fq,
                     const float *fF, long long frame0, long long n_avail, int n_frames, cudaStream_t s) {
    if (t.N > kTrainMaxN || P.n_layers != 1 || P.n_ang != 0 || t.W > 32) return LSD_EUNSUPPORTED;
    int r = ensure_frame_bufs(t, n_frames);
    if (r != LSD_OK) return r;
    const TrainGeo T = make_tgeo(t, P);
    const float scale = -2.0f / ((float)n_frames * 3.0f * (float)t.N);
    fm_frame_kernel<<<n_frames, kTrainThreads, fm_smem(t), s>>>(T, g, P, t.w, species, fq, fF, frame0, n_avail, scale,
                                                               t.grad_frames, t.loss_frames);
    const int nw = (int)t.n_weights;
    fm_reduce_kernel<<<(nw + 255) / 256, 256, 0, s>>>(t.grad_frames, t.loss_frames, n_frames, nw, t.grad, t.loss);
    return cudaGetLastError() == cudaSuccess ? LSD_OK : LSD_ECUDA;
}

int train_force_match(TrainState &t, const Geo &g, const PotDev &P, const int *species, const double *fq,
                      const float *fF, int n_frames, float *loss_out, float *grad_dev, cudaStream_t s) {
    if (!t.enabled) return LSD_EINVAL;
    int r = fm_launch(t, g, P, species, fq, fF, 0, n_frames, n_frames, s);
    if (r != LSD_OK) return r;
    if (grad_dev &&
        cudaMemcpyAsync(grad_dev, t.grad, t.n_weights * sizeof(float), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return LSD_ECUDA;
    float l = 0.f;
    if (cudaMemcpyAsync(&l, t.loss, sizeof(float), cudaMemcpyDeviceToHost, s) != cudaSuccess) return LSD_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return LSD_ECUDA;
    if (loss_out) *loss_out = l;
    return LSD_OK;
}

int train_run(TrainState &t, const Geo &g, const PotDev &P, const int *species, int n_iters, float lr,
              int frames_per_iter, float *loss_out, cudaStream_t s) {
    if (!t.enabled) return LSD_EINVAL;
    int64_t avail = 0;
    int r = train_frame_count(t, &avail, s);
    if (r != LSD_OK) return r;
    if (avail < 1) return LSD_ESTATE;
    const int fpi = (frames_per_iter <= 0 || frames_per_iter > avail) ? (int)avail : frames_per_iter;
    const int nw = (int)t.n_weights;
    for (int it = 0; it < n_iters; ++it) {
        const long long frame0 = (t.iter * (long long)fpi) % avail;
        r = fm_launch(t, g, P, species, t.fq, t.fF, frame0, avail, fpi, s);
        if (r != LSD_OK) return r;
        ++t.adam_t;
        ++t.iter;
        const float b1 = 0.9f, b2 = 0.999f;
        const float c1 = 1.f - powf(b1, (float)t.adam_t), c2 = 1.f - powf(b2, (float)t.adam_t);
        adam_kernel<<<(nw + 255) / 256, 256, 0, s>>>(t.w, t.m, t.v, t.grad, nw, lr, b1, b2, 1e-8f, c1, c2);
    }
    if (loss_out) {
        float l = 0.f;
        if (cudaMemcpyAsync(&l, t.loss, sizeof(float), cudaMemcpyDeviceToHost, s) != cudaSuccess) return LSD_ECUDA;
        if (cudaStreamSynchronize(s) != cudaSuccess) return LSD_ECUDA;
        *loss_out = l;
    }
    return cudaStreamSynchronize(s) == cudaSuccess ? LSD_OK : LSD_ECUDA;
}

}  // namespace lsd
