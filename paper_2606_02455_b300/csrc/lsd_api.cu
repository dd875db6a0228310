// lsd_api.cu -- host side of the C ABI declared in include/lsd.h.
//
// A handle owns all device memory of one simulation: the base state (FP64),
// the window arrays of K drafted steps, the batched-verification workspace
// (K*N rows), the device-resident run state, and two CUDA graphs: one window
// (draft -> batched target forces -> transport/commit) and one plain target
// step.  lsd_step replays the window graph without reading anything back per
// window: every kernel reads the step counter and the stop step from device
// memory and turns itself into a no-op once enough steps are committed, so
// the host only synchronises once per batch of windows.
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstddef>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "lsd.h"
#include "lsd_common.cuh"
#include "lsd_kernels.h"
#include "lsd_train.h"

using namespace lsd;

namespace {

constexpr double kTwo32 = 4294967296.0;
constexpr int kMaxDynSmem = 227 * 1024;
constexpr double kWaitLimitSeconds = 600.0;
constexpr double kMomMinNeighbours = 40.0;   // expected descriptor neighbours per atom from which moments are used

double kappa_conv() { return (1.602176634e-19 / 1e-10) / (1.66053906660e-27 * 1e-10 / 1e-30); }
double kboltz_ev() { return 1.380649e-23 / 1.602176634e-19; }

struct PotHost {
    lsd_potential p{};
    std::vector<double> eps, sigma;
    std::vector<float> weights;
    PotDev dev{};
    float *dbuf = nullptr;            // Wt, Wn, b, wout (FP32)
    __nv_bfloat16 *dbuf_bf = nullptr; // Wt, Wn, wout (BF16)
    float rmax2f = 0.f, near2f = 0.f;
    bool present = false;
    void *tc_plan = nullptr;              // tensor maps of the weights (tensor-core MLP: BF16, TF32x3 or FP8)
    void *cal_plan = nullptr;             // FP8: the BF16 plan that calibrates the activation scales
    __nv_bfloat16 *tc_scratch = nullptr;  // per-CTA SiLU' slots of the tensor-core MLP (when not in TMEM)
    size_t n_dbuf = 0;                    // floats in dbuf
    float *dbuf_tf = nullptr;             // TF32 hi parts of the FP32 layouts, then the lo parts
    __half *dbuf_h = nullptr;             // scaled FP16 hi parts of the FP32 layouts, then the lo parts
    uint8_t *dbuf_f8 = nullptr;           // e4m3 copies of the FP32 layouts (per-layer scales)
    float *tc_scales = nullptr;           // FP8, F16x3 [3L]: forward A, backward A, weight dequantisation factors
    float *tc_amax = nullptr;             // calibration [2L]
};

}  // namespace

struct lsd_handle {
    int dev = 0;
    int n_sm = 148;
    int N = 0, S = 0, K = 0;
    double box[3] = {0, 0, 0};
    double gamma = 0, dt = 0, T = 0;
    uint64_t seed = 0;
    std::vector<int> species_h;
    std::vector<double> mass_h;
    Geo geo{};
    Coef coef{};
    double *p_obabo = nullptr;   // OBABO output momenta of the current step (staggered frame: p is the staggered one)
    PotHost draft, target;
    bool learned_small = false;
    DraftPlan dplan{};
    bool mom_on = false;            // the target's angular features and adjoint by moments
    float *mom = nullptr;           // their per-row moments [K N][kMomRowFloats]
    DraftPlan gplan{};              // the grid form of the draft (large systems), when the device co-schedules it
    DraftPlan dplan0{}, gplan0{};   // both as planned for windows of K steps
    bool grid_draft = false;        // windows and redrafts draft in the grid form
    DraftSync *dsync = nullptr;     // its barrier and flag words
    VerletPlan vplan{};
    VerletBufs vbufs{};
    float *w_dEdX = nullptr;
    int *w_nbr = nullptr;   // learned draft: each atom's neighbours within its largest cutoff [N][nbr_cap], counts [N]
    int nbr_cap = 0;
    // device state
    double *q = nullptr, *p = nullptr;
    int *species = nullptr;
    DevState *st = nullptr;
    // window arrays
    double *w_qmid = nullptr, *w_pdraft = nullptr;
    float *w_Fd = nullptr, *w_Fraw = nullptr, *w_Ft = nullptr;
    uint4 *w_fix = nullptr, *fix_eval = nullptr;
    float *ec_dF = nullptr;
    int ec_on = 0;
    // verification workspace (M = K*N rows)
    int cap_near = 0, cap_far = 0;
    int *near_keys = nullptr, *far_keys = nullptr, *n_near = nullptr, *n_far = nullptr;
    float *X = nullptr, *dEdX = nullptr, *E_mlp = nullptr, *E_lj = nullptr, *E_atom = nullptr;
    float4 *pair_g = nullptr, *Fpart = nullptr;
    double2 *partials = nullptr;
    // streams and graphs
    cudaStream_t own_stream = nullptr, stream = nullptr;
    cudaGraphExec_t g_window = nullptr, g_plain = nullptr;
    // the pipelined window loop: two window buffers (buffer 0 aliases the
    // per-window arrays above), their headers, the speculative base state, a
    // high-priority draft stream and the fork/join events of a round
    struct WinBufs {
        double *qmid = nullptr, *pdraft = nullptr;
        float *Fd = nullptr, *Fraw = nullptr;
        uint4 *fix = nullptr;
        VerletBufs vb;
    } wb[2];
    bool pipe_on = false, pipe_alloc = false, pipe_primed = false;
    int pipe_cur = 0;
    WinHdr *hdr = nullptr;
    double *qb = nullptr, *pb = nullptr;
    cudaStream_t dstream = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_v = nullptr, ev_d = nullptr;
    cudaEvent_t ev_sync = nullptr;   // wait_stream's event, created once
    cudaGraphExec_t g_round[2] = {nullptr, nullptr};
    float move2f_list = 0.f;   // (0.45 skin)^2: the largest displacement the lists stay complete for
    float move2f_user = 0.f;   // lsd_set_max_displacement's bound squared (0: none)
    double list_rcut = 0.0, list_skin0 = 0.0, list_skin = 0.0;   // the lists' cutoff, planned and current skin
    // online retraining of a learned draft (lsd_set_online_training)
    long long online_every = 0;        // accepted steps between retrainings (0: off)
    int online_iters = 0, online_fpi = 0;
    float online_lr = 0.f;
    long long online_base = 0;         // accepted-step count at the last retraining
    long long online_count = 0;
    float online_loss = 0.f;
    // the fused plain-target step (small FP32 targets): plan, whether it is in use, exchange buffers
    PlainPlan pplan{};
    bool plain_fused = false;
    uint4 *pf_fix = nullptr;
    int *pf_keys = nullptr, *pf_cnt = nullptr;
    float4 *pf_pg = nullptr;
    unsigned long long *pf_bar = nullptr;   // its grid-barrier counter
    int stage_len = 0;        // windows verified in stages of this many steps (0: in one pass)
    bool pdl_graphs = true;   // the captured graphs' kernels overlap their predecessors' tails (small systems)
    bool list_reuse = false;  // unpipelined windows keep their Verlet lists while the committed state stays close
    bool drafted = false;
    bool unbounded = false;   // target_step set to "no cap" by lsd_enqueue_*
    // learned-draft training
    TrainState train{};
    std::vector<void *> allocs;
};

namespace {

cudaError_t g_last_cuda = cudaSuccess;

#define CK(x)                                   \
    do {                                        \
        cudaError_t e_ = (x);                   \
        if (e_ != cudaSuccess) {                \
            g_last_cuda = e_;                   \
            return LSD_ECUDA;                   \
        }                                       \
    } while (0)

template <typename T>
int dalloc(lsd_handle *h, T **ptr, size_t count) {
    *ptr = nullptr;
    if (count == 0) count = 1;
    void *v = nullptr;
    cudaError_t e = cudaMalloc(&v, count * sizeof(T));
    if (e != cudaSuccess) {
        g_last_cuda = e;
        return LSD_ENOMEM;
    }
    cudaMemset(v, 0, count * sizeof(T));
    h->allocs.push_back(v);
    *ptr = (T *)v;
    return LSD_OK;
}

#define TRY(x)                   \
    do {                         \
        int r_ = (x);            \
        if (r_ != LSD_OK) return r_; \
    } while (0)

int input_dim(int S, int nr, int na) { return S * nr + na + S; }

size_t n_weights(int d0, int L, int W) {
    if (L <= 0) return 0;
    return (size_t)W * d0 + W + (size_t)(L - 1) * ((size_t)W * W + W) + W + 1;
}

int pot_setup(lsd_handle *h, PotHost &ph, const lsd_potential *lp, bool is_draft) {
    if (!lp) return LSD_EINVAL;
    ph.p = *lp;
    ph.present = true;
    const int S = h->S;
    const double bmin = std::min(h->box[0], std::min(h->box[1], h->box[2]));
    PotDev &P = ph.dev;
    P = PotDev{};
    P.kind = lp->kind;
    P.precision = lp->precision;
    P.head = lp->head;
    P.head_scale = (float)lp->head_scale;
    if (lp->kind < LSD_POT_LJ || lp->kind > LSD_POT_LEARNED) return LSD_EINVAL;
    if (lp->precision < LSD_FP32 || lp->precision > LSD_FP32_TF32) return LSD_EINVAL;
    P.has_lj = lp->lj_cutoff > 0.0;
    P.has_mlp = lp->kind != LSD_POT_LJ && lp->n_layers > 0;
    if (P.has_lj) {
        if (!lp->lj_eps || !lp->lj_sigma) return LSD_EINVAL;
        if (!(lp->lj_cutoff < bmin)) return LSD_EINVAL;
        ph.eps.assign(lp->lj_eps, lp->lj_eps + S);
        ph.sigma.assign(lp->lj_sigma, lp->lj_sigma + S);
        const double rc = lp->lj_cutoff;
        P.lj_rc2f = (float)(rc * rc);
        for (int a = 0; a < S; ++a)
            for (int b = 0; b < S; ++b) {
                const double e = std::sqrt(ph.eps[a] * ph.eps[b]);
                const double s = 0.5 * (ph.sigma[a] + ph.sigma[b]);
                const double sc6 = std::pow(s / rc, 6.0);
                P.lj_sig2[a * S + b] = (float)(s * s);
                P.lj_eps24[a * S + b] = (float)(24.0 * e);
                P.lj_eps4[a * S + b] = (float)(4.0 * e);
                P.lj_shift[a * S + b] = (float)(4.0 * e * (sc6 * sc6 - sc6));
            }
    }
    if (P.has_mlp) {
        const double rc = lp->desc_cutoff;
        if (!(rc > 0.0) || !(rc < bmin)) return LSD_EINVAL;
        if (lp->n_rbf < 2 || lp->n_rbf > 16) return LSD_EINVAL;
        if (lp->n_ang != 0 && lp->n_ang != kNAng) return LSD_EINVAL;
        if (lp->n_layers < 1 || lp->n_layers > kMaxLayers) return LSD_EINVAL;
        if (lp->width < 32 || lp->width > 256 || lp->width % 32) return LSD_EUNSUPPORTED;
        if (lp->head != LSD_HEAD_TANH && lp->head != LSD_HEAD_LINEAR) return LSD_EINVAL;
        if (lp->kind == LSD_POT_LEARNED && lp->head != LSD_HEAD_LINEAR) return LSD_EINVAL;
        P.n_rbf = lp->n_rbf;
        P.n_ang = lp->n_ang;
        P.n_layers = lp->n_layers;
        P.width = lp->width;
        P.d0 = input_dim(S, lp->n_rbf, lp->n_ang);
        P.d0p = (P.d0 + 31) / 32 * 32;
        P.desc_rc = (float)rc;
        P.desc_rc2f = (float)(rc * rc);
        const double w = rc / (double)(lp->n_rbf - 1);
        P.rbf_w = (float)w;
        P.rbf_inv2w2 = (float)(1.0 / (2.0 * w * w));
        P.rbf_invw2 = (float)(1.0 / (w * w));
        const size_t nw = n_weights(P.d0, P.n_layers, P.width);
        if (!lp->weights || lp->n_weights != nw) return LSD_EINVAL;
        ph.weights.assign(lp->weights, lp->weights + nw);
        // device layouts: Wt[l] [din_p][W], Wn[l] [W][din_p], b[l] [W], wout [W]
        const int W = P.width, L = P.n_layers;
        size_t total = 0;
        std::vector<size_t> offWt(L), offWn(L), offb(L);
        for (int l = 0; l < L; ++l) {
            const int dinp = l == 0 ? P.d0p : W;
            offWt[l] = total; total += (size_t)dinp * W;
            offWn[l] = total; total += (size_t)dinp * W;
            offb[l] = total; total += W;
        }
        const size_t offwo = total;
        total += W;
        ph.n_dbuf = total;
        TRY(dalloc(h, &ph.dbuf, total));
        TRY(dalloc(h, &ph.dbuf_bf, total));
        if (lp->precision == LSD_FP32 || lp->precision == LSD_FP32_TF32) TRY(dalloc(h, &ph.dbuf_tf, 2 * total));
        if (lp->precision == LSD_FP32) {
            TRY(dalloc(h, &ph.dbuf_h, 2 * total));
            TRY(dalloc(h, &ph.tc_scales, 3 * (size_t)L));
            TRY(dalloc(h, &ph.tc_amax, 2 * (size_t)L));
        }
        if (lp->precision == LSD_FP8) {
            TRY(dalloc(h, &ph.dbuf_f8, total));
            TRY(dalloc(h, &ph.tc_scales, 3 * (size_t)L));
            TRY(dalloc(h, &ph.tc_amax, 2 * (size_t)L));
        }
        for (int l = 0; l < L; ++l) {
            P.Wt[l] = ph.dbuf + offWt[l];
            P.Wn[l] = ph.dbuf + offWn[l];
            P.b[l] = ph.dbuf + offb[l];
            P.Wt_bf[l] = ph.dbuf_bf + offWt[l];
            P.Wn_bf[l] = ph.dbuf_bf + offWn[l];
        }
        P.wout = ph.dbuf + offwo;
        P.wout_bf = ph.dbuf_bf + offwo;
        if (is_draft && lp->kind == LSD_POT_LEARNED) {
            if (P.n_layers != 1 || P.width > 32 || P.n_ang != 0 || P.d0p > 32) return LSD_EUNSUPPORTED;
        }
    }
    ph.rmax2f = std::max(P.lj_rc2f, P.desc_rc2f);
    P.rmax2f = ph.rmax2f;   // the fused plain step reads it from the potential block
    ph.near2f = P.has_mlp ? P.desc_rc2f : 0.f;
    return LSD_OK;
}

// Uploads ph.weights into the device layouts (FP32 and BF16).
int pot_upload(lsd_handle *h, PotHost &ph) {
    PotDev &P = ph.dev;
    if (!P.has_mlp) return LSD_OK;
    const int W = P.width, L = P.n_layers;
    std::vector<float> buf;
    std::vector<size_t> offWt(L), offWn(L), offb(L);
    size_t total = 0;
    for (int l = 0; l < L; ++l) {
        const int dinp = l == 0 ? P.d0p : W;
        offWt[l] = total; total += (size_t)dinp * W;
        offWn[l] = total; total += (size_t)dinp * W;
        offb[l] = total; total += W;
    }
    const size_t offwo = total;
    total += W;
    buf.assign(total, 0.f);
    const float *w = ph.weights.data();
    for (int l = 0; l < L; ++l) {
        const int din = l == 0 ? P.d0 : W, dinp = l == 0 ? P.d0p : W;
        for (int o = 0; o < W; ++o)
            for (int k = 0; k < din; ++k) {
                const float v = w[(size_t)o * din + k];
                buf[offWt[l] + (size_t)k * W + o] = v;
                buf[offWn[l] + (size_t)o * dinp + k] = v;
            }
        w += (size_t)W * din;
        for (int o = 0; o < W; ++o) buf[offb[l] + o] = w[o];
        w += W;
    }
    for (int o = 0; o < W; ++o) buf[offwo + o] = w[o];
    P.bout = w[W];
    std::vector<__nv_bfloat16> bb(total);
    for (size_t k = 0; k < total; ++k) bb[k] = __float2bfloat16(buf[k]);
    CK(cudaMemcpyAsync(ph.dbuf, buf.data(), total * sizeof(float), cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(ph.dbuf_bf, bb.data(), total * sizeof(__nv_bfloat16), cudaMemcpyHostToDevice, h->stream));
    std::vector<float> tf;
    if (ph.dbuf_tf) {
        // TF32 split, round to nearest with ties away from zero on the magnitude
        // (the low 13 of 23 fraction bits dropped): hi = tf32(w), lo = tf32(w - hi)
        auto tf32 = [](float x) {
            uint32_t u;
            std::memcpy(&u, &x, 4);
            if ((u & 0x7f800000u) != 0x7f800000u) u = (u + 0x1000u) & 0xffffe000u;
            float r;
            std::memcpy(&r, &u, 4);
            return r;
        };
        tf.resize(2 * total);
        for (size_t k = 0; k < total; ++k) {
            tf[k] = tf32(buf[k]);
            tf[total + k] = tf32(buf[k] - tf[k]);
        }
        CK(cudaMemcpyAsync(ph.dbuf_tf, tf.data(), 2 * total * sizeof(float), cudaMemcpyHostToDevice, h->stream));
    }
    std::vector<__half> hh;
    std::vector<float> hsc;
    if (ph.dbuf_h) {
        // FP16 split of W s_l, s_l = 2^(14 - ceil log2 max|W_l|) (exact): hi = fp16(W s), lo = fp16(W s - hi)
        hh.resize(2 * total);
        hsc.assign(L, 1.f);
        for (int l = 0; l < L; ++l) {
            const int dinp = l == 0 ? P.d0p : W;
            float m = 0.f;
            for (size_t k = 0; k < (size_t)dinp * W; ++k) m = std::max(m, std::fabs(buf[offWn[l] + k]));
            const float sc = m > 0.f ? std::ldexp(1.f, 14 - (int)std::ceil(std::log2(m))) : 1.f;
            hsc[l] = 1.f / sc;
            for (const size_t off : {offWn[l], offWt[l]})
                for (size_t k = 0; k < (size_t)dinp * W; ++k) {
                    const float x = buf[off + k] * sc;
                    const __half hi = __float2half_rn(x);
                    hh[off + k] = hi;
                    hh[total + off + k] = __float2half_rn(x - __half2float(hi));
                }
        }
        CK(cudaMemcpyAsync(ph.dbuf_h, hh.data(), 2 * total * sizeof(__half), cudaMemcpyHostToDevice, h->stream));
        CK(cudaMemcpyAsync(ph.tc_scales + 2 * L, hsc.data(), L * sizeof(float), cudaMemcpyHostToDevice, h->stream));
    }
    std::vector<uint8_t> f8;
    std::vector<float> wsc;
    if (ph.dbuf_f8) {
        // e4m3 with one scale per layer: s_l = max|W_l| / 448 (the largest finite e4m3), both layouts
        f8.assign(total, 0);
        wsc.assign(L, 1.f);
        for (int l = 0; l < L; ++l) {
            const int dinp = l == 0 ? P.d0p : W;
            float m = 0.f;
            for (size_t k = 0; k < (size_t)dinp * W; ++k) m = std::max(m, std::fabs(buf[offWn[l] + k]));
            wsc[l] = m > 0.f ? m / 448.f : 1.f;
            for (size_t k = 0; k < (size_t)dinp * W; ++k) {
                f8[offWn[l] + k] = __nv_cvt_float_to_fp8(buf[offWn[l] + k] / wsc[l], __NV_SATFINITE, __NV_E4M3);
                f8[offWt[l] + k] = __nv_cvt_float_to_fp8(buf[offWt[l] + k] / wsc[l], __NV_SATFINITE, __NV_E4M3);
            }
        }
        CK(cudaMemcpyAsync(ph.dbuf_f8, f8.data(), total, cudaMemcpyHostToDevice, h->stream));
        CK(cudaMemcpyAsync(ph.tc_scales + 2 * L, wsc.data(), L * sizeof(float), cudaMemcpyHostToDevice, h->stream));
    }
    CK(cudaStreamSynchronize(h->stream));
    return LSD_OK;
}

int nb_capacity(double density, double rc, int extra) {
    const double expect = density * 4.0 / 3.0 * 3.14159265358979 * rc * rc * rc;
    int cap = (int)std::ceil(2.0 * expect) + extra;
    return (cap + 31) / 32 * 32;
}

int wait_stream(lsd_handle *h) {
    if (!h->ev_sync) CK(cudaEventCreateWithFlags(&h->ev_sync, cudaEventDisableTiming));
    cudaError_t e = cudaEventRecord(h->ev_sync, h->stream);
    if (e != cudaSuccess) {
        g_last_cuda = e;
        return LSD_ECUDA;
    }
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        e = cudaEventQuery(h->ev_sync);
        if (e == cudaSuccess) break;
        if (e != cudaErrorNotReady) {
            g_last_cuda = e;
            return LSD_ECUDA;
        }
        const double dtw = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (dtw > kWaitLimitSeconds) return LSD_ETIMEOUT;
    }
    return LSD_OK;
}

// The MLP of a batched evaluation: tcgen05 tensor cores for BF16 potentials,
// the FP32 CUDA-core kernel otherwise.
void enqueue_mlp(lsd_handle *h, const PotHost &pot, int M, cudaStream_t s) {
    const PotDev &P = pot.dev;
    if (pot.tc_plan)
        launch_mlp_tc(pot.tc_plan, h->X, M, P, h->E_mlp, h->dEdX, pot.tc_scratch, pot.tc_scales, nullptr, h->n_sm,
                      &h->st->err, s);
    else
        launch_mlp_fp32(h->X, M, P, h->E_mlp, h->dEdX, s);
}

// The moment buffer when pot's angular block runs by moments (the target, with
// rows dense enough), else null.
float *mom_for(const lsd_handle *h, const PotHost &pot) {
    return (h->mom_on && &pot == &h->target && pot.dev.n_ang) ? h->mom : nullptr;
}

// Batched force evaluation of `pot` on Kc configurations whose fixed-point
// coordinates are in fix ([Kc][N]); forces to F ([Kc][N][3]).
// With use_list the candidates are the window's Verlet lists (the window and
// plain-step paths); otherwise all atoms (explicit configurations).
// j_off: the window step of row block 0 (one stage of a window verified in
// stages), against which keff is compared.
void enqueue_eval(lsd_handle *h, const PotHost &pot, const uint4 *fix, int Kc, float *F, float *E_out,
                  cudaStream_t s, bool use_list = false, const VerletBufs *vb = nullptr, const int *keff = nullptr,
                  int j_off = 0) {
    const int M = Kc * h->N;
    const PotDev &P = pot.dev;
    if (!vb) vb = &h->vbufs;
    const int *keff_rows = keff;   // window paths: rows past the draft's k_eff stay empty (null: every row)
    if (!keff) keff = &h->st->k_eff;
    if (use_list)
        launch_neigh_list(fix, vb->vlist, vb->vcount, h->vplan.cap, M, h->geo, pot.rmax2f, pot.near2f,
                          h->cap_near, h->cap_far, h->near_keys, h->far_keys, h->n_near, h->n_far, h->st, keff, s,
                          j_off);
    else
        launch_neigh_build(fix, M, h->geo, pot.rmax2f, pot.near2f, h->cap_near, h->cap_far, h->near_keys,
                           h->far_keys, h->n_near, h->n_far, h->st, s, keff_rows, j_off);
    if (P.has_mlp) {
        launch_desc(fix, h->near_keys, h->n_near, h->cap_near, M, h->geo, P, h->X, s, mom_for(h, pot));
        enqueue_mlp(h, pot, M, s);
    }
    launch_pairgrad(fix, h->near_keys, h->n_near, h->far_keys, h->n_far, h->cap_near, h->cap_far, M, h->geo, P, h->dEdX,
                    h->pair_g, h->Fpart, h->E_lj, s, mom_for(h, pot));
    launch_force_gather(h->near_keys, h->n_near, h->cap_near, M, h->N, P.has_mlp, h->pair_g, h->Fpart, h->E_lj,
                        h->E_mlp, F, E_out, h->st, s);
}

// Lists kept across windows (lsd_set_list_reuse): rebuilt around the
// committed state only when some atom has moved more than half the draft's
// displacement bound from their base, or the last draft stopped at the bound.
void enqueue_kept_lists(lsd_handle *h, lsd_handle::WinBufs &w, cudaStream_t s) {
    launch_verlet_check(h->q, w.vb, h->geo, 0.25f * h->vplan.move2f, h->st, s);
    launch_verlet_build(h->vplan, h->q, h->species, h->geo, w.vb, h->st, s, nullptr, &h->st->list_rebuild);
}

// The window's Verlet lists around the base state, then the draft, into
// window buffer b.  hdr null: from the committed state (q, p, st->step);
// else (pipelined loop) from the base (q, p) at step hdr->base, skipped when
// hdr->skip is set.
void enqueue_draft_buf(lsd_handle *h, int b, cudaStream_t s, WinHdr *hdr, const double *q, const double *p,
                       bool redraft = false, int Kd = 0) {   // Kd: steps to draft (0: the window's K)
    lsd_handle::WinBufs &w = h->wb[b];
    if (!h->vplan.all_pairs) {
        if (redraft) launch_redraft_flag(h->st, hdr, s);
        if (!hdr && h->list_reuse) {
            enqueue_kept_lists(h, w, s);
        } else {
            launch_verlet_build(h->vplan, q, h->species, h->geo, w.vb, h->st, s,
                                hdr ? (redraft ? &hdr->keep : &hdr->skip) : nullptr);
        }
    }
    // the speculative draft of the pipelined loop overlaps a verification: the cluster form, on a few SMs
    const bool grid = h->grid_draft && (!hdr || redraft);
    launch_draft(grid ? h->gplan : h->dplan, h->learned_small, Kd ? Kd : h->K, h->geo, h->draft.dev, h->coef, h->vplan, w.vb,
                 h->species, q, p, h->ec_dF, h->ec_on, h->st, w.qmid, w.pdraft, w.Fd, w.Fraw, w.fix, h->w_dEdX, s, hdr,
                 redraft ? 1 : 0, h->dsync, 0, h->w_nbr, h->nbr_cap);
}

// Verification, frames and transport of window buffer b; keff: the window's
// drafted step count (its header in a pipelined round, else the run state's).
void enqueue_verify_buf(lsd_handle *h, int b, cudaStream_t s, const int *keff) {
    lsd_handle::WinBufs &w = h->wb[b];
    enqueue_eval(h, h->target, w.fix, h->K, h->w_Ft, nullptr, s, !h->vplan.all_pairs, &w.vb, keff);
    if (h->train.capture_on) enqueue_frame_capture(h->train, w.qmid, h->w_Ft, h->K, h->N, h->st, keff, s);
    launch_transport(h->K, h->geo, h->coef, h->species, w.qmid, w.pdraft, w.Fd, h->w_Ft, w.Fraw, h->ec_dF, h->ec_on,
                     h->q, h->p, h->p_obabo, h->st, h->partials, keff, s);
}

// Stage [j0, j1) of a window verified in stages: the Verlet lists (first
// stage), the draft of steps j0 .. j1 - 1 continued from step j0 - 1, their
// verification in rows 0 .. j1 - j0 - 1 of the workspace, and the transport's
// decision over steps 0 .. j1 - 1.  next: the conditional handle of the next
// stage's node (0 for the last stage), set by the transport when the window
// goes on.
void enqueue_stage(lsd_handle *h, int j0, int j1, cudaGraphConditionalHandle next, cudaStream_t s) {
    lsd_handle::WinBufs &w = h->wb[0];
    const size_t N = h->N;
    const int *keff = &h->st->k_eff;
    if (j0 == 0 && !h->vplan.all_pairs) {
        if (h->list_reuse)
            enqueue_kept_lists(h, w, s);
        else
            launch_verlet_build(h->vplan, h->q, h->species, h->geo, w.vb, h->st, s);
    }
    launch_draft(h->grid_draft ? h->gplan : h->dplan, h->learned_small, j1, h->geo, h->draft.dev, h->coef, h->vplan,
                 w.vb, h->species, h->q, h->p, h->ec_dF, h->ec_on, h->st, w.qmid, w.pdraft, w.Fd, w.Fraw, w.fix,
                 h->w_dEdX, s, nullptr, 0, h->dsync, j0, h->w_nbr, h->nbr_cap);
    enqueue_eval(h, h->target, w.fix + (size_t)j0 * N, j1 - j0, h->w_Ft + (size_t)j0 * 3 * N, nullptr, s,
                 !h->vplan.all_pairs, &w.vb, keff, j0);
    if (h->train.capture_on) enqueue_frame_capture(h->train, w.qmid, h->w_Ft, j1, h->N, h->st, keff, s, j0);
    launch_transport(j1, h->geo, h->coef, h->species, w.qmid, w.pdraft, w.Fd, h->w_Ft, w.Fraw, h->ec_dF, h->ec_on,
                     h->q, h->p, h->p_obabo, h->st, h->partials, keff, s, j0, next ? 1 : 0, next);
}

void enqueue_draft(lsd_handle *h, cudaStream_t s) { enqueue_draft_buf(h, 0, s, nullptr, h->q, h->p); }
void enqueue_verify(lsd_handle *h, cudaStream_t s) { enqueue_verify_buf(h, 0, s, &h->st->k_eff); }

// One round of the pipelined loop: verify window b on the main stream while
// the draft stream drafts window b^1 speculatively; then keep or redraft b^1.
void enqueue_round(lsd_handle *h, int b) {
    cudaStream_t V = h->stream, D = h->dstream;
    const int n = b ^ 1;
    cudaEventRecord(h->ev_fork, V);
    cudaStreamWaitEvent(D, h->ev_fork, 0);
    enqueue_verify_buf(h, b, V, &h->hdr[b].k_eff);
    launch_spec_base(h->geo, h->coef, h->species, h->wb[b].qmid, h->wb[b].pdraft, &h->hdr[b], &h->hdr[n], h->st,
                     h->qb, h->pb, D);
    enqueue_draft_buf(h, n, D, &h->hdr[n], h->qb, h->pb);
    cudaEventRecord(h->ev_v, V);
    cudaStreamWaitEvent(D, h->ev_v, 0);
    enqueue_draft_buf(h, n, D, &h->hdr[n], h->q, h->p, true);   // returns at once when the speculative draft stands
    cudaEventRecord(h->ev_d, D);
    cudaStreamWaitEvent(V, h->ev_d, 0);
}

// The first window of a pipelined run: drafted from the committed state into buffer 0.
void enqueue_prime(lsd_handle *h) {
    launch_hdr_invalidate(&h->hdr[0], h->stream);
    enqueue_draft_buf(h, 0, h->stream, &h->hdr[0], h->q, h->p, true);
    h->pipe_primed = true;
    h->pipe_cur = 0;
}

// One plain target step.  Its Verlet lists are kept from step to step while
// the evaluated (half-step) positions stay within the displacement bound of
// their base, the draft's criterion, and rebuilt around those positions
// otherwise: every pair within the cutoff is listed either way, and the
// neighbour keys are sorted, so the forces do not depend on which lists hold
// them.
void enqueue_plain(lsd_handle *h, cudaStream_t s) {
    launch_plain_half(h->geo, h->coef, h->species, h->q, h->p, h->st, h->w_qmid, h->w_fix, s);
    if (!h->vplan.all_pairs) {
        launch_verlet_check(h->w_qmid, h->vbufs, h->geo, h->vplan.move2f, h->st, s);
        launch_verlet_build(h->vplan, h->w_qmid, h->species, h->geo, h->vbufs, h->st, s, nullptr,
                            &h->st->list_rebuild);
    }
    enqueue_eval(h, h->target, h->w_fix, 1, h->w_Ft, nullptr, s, !h->vplan.all_pairs);
    launch_plain_finish(h->geo, h->coef, h->species, h->w_qmid, h->w_Ft, h->q, h->p, h->p_obabo, h->st, s);
}

// n plain target steps in one launch of the fused kernel (ABOBA only).
bool use_plain_fused(const lsd_handle *h) { return h->plain_fused && !h->coef.obabo; }

int launch_plain_steps_fused(lsd_handle *h, long long n) {
    while (n > 0) {
        const int chunk = n > (1 << 30) ? (1 << 30) : (int)n;
        CK(launch_plain_fused(h->pplan, chunk, h->geo, h->target.dev, h->coef, h->species, h->q, h->p, h->pf_fix,
                              h->pf_keys, h->pf_cnt, h->pf_pg, h->pf_bar, h->st, h->stream));
        n -= chunk;
    }
    return LSD_OK;
}

void destroy_graphs(lsd_handle *h) {
    if (h->g_window) cudaGraphExecDestroy(h->g_window);
    if (h->g_plain) cudaGraphExecDestroy(h->g_plain);
    h->g_window = h->g_plain = nullptr;
    for (auto &g : h->g_round) {
        if (g) cudaGraphExecDestroy(g);
        g = nullptr;
    }
    h->pipe_primed = false;   // a later pipelined run drafts its first window afresh
}

// Sets whether the launches captured into a graph are programmatic dependent
// launches (the handle's choice), for the scope of one capture.
struct PdlScope {
    int saved;
    explicit PdlScope(const lsd_handle *h) : saved(pdl_current()) { pdl_current() = h->pdl_graphs ? 1 : 0; }
    ~PdlScope() { pdl_current() = saved; }
};

int build_graph(lsd_handle *h, void (*fn)(lsd_handle *, cudaStream_t), cudaGraphExec_t *out) {
    PdlScope pdl(h);
    cudaGraph_t g;
    CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    fn(h, h->stream);
    CK(cudaStreamEndCapture(h->stream, &g));
    cudaError_t e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    CK(e);
    return LSD_OK;
}

void window_fn(lsd_handle *h, cudaStream_t s) {
    enqueue_draft(h, s);
    enqueue_verify(h, s);
}

int build_round_graph(lsd_handle *h, int b, cudaGraphExec_t *out) {
    PdlScope pdl(h);
    cudaGraph_t g;
    CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    enqueue_round(h, b);
    CK(cudaStreamEndCapture(h->stream, &g));
    cudaError_t e = cudaGraphInstantiate(out, g, cudaGraphInstantiateFlagUseNodePriority);
    cudaGraphDestroy(g);
    CK(e);
    return LSD_OK;
}

// A window verified in stages of stage_len steps: stage 0 in the top graph,
// then stage s in the body of an IF node that follows stage s - 1's transport
// (nested: each handle belongs to the graph whose kernel sets it).
int build_staged_graph(lsd_handle *h, cudaGraphExec_t *out) {
    PdlScope pdl(h);
    const int K = h->K, S = h->stage_len, n_stages = (K + S - 1) / S;
    cudaGraph_t top = nullptr;
    CK(cudaGraphCreate(&top, 0));
    cudaGraph_t cur = top;
    cudaError_t e = cudaSuccess;
    for (int st = 0; st < n_stages && e == cudaSuccess; ++st) {
        const int j0 = st * S, j1 = j0 + S < K ? j0 + S : K;
        const bool more = st + 1 < n_stages;
        cudaGraphConditionalHandle next = 0;
        if (more && (e = cudaGraphConditionalHandleCreate(&next, cur, 0u, cudaGraphCondAssignDefault)) != cudaSuccess)
            break;
        if ((e = cudaStreamBeginCaptureToGraph(h->stream, cur, nullptr, nullptr, 0,
                                               cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
            break;
        enqueue_stage(h, j0, j1, next, h->stream);
        cudaGraph_t body = nullptr;
        if (more) {
            cudaStreamCaptureStatus cs;
            cudaGraph_t cg = nullptr;
            const cudaGraphNode_t *deps = nullptr;
            const cudaGraphEdgeData *edges = nullptr;
            size_t n_deps = 0;
            e = cudaStreamGetCaptureInfo(h->stream, &cs, nullptr, &cg, &deps, &edges, &n_deps);
            edges = nullptr;   // the IF node follows its predecessors with full serialisation
            if (e == cudaSuccess) {
                cudaGraphNodeParams np = {};
                np.type = cudaGraphNodeTypeConditional;
                np.conditional.handle = next;
                np.conditional.type = cudaGraphCondTypeIf;
                np.conditional.size = 1;
                cudaGraphNode_t node;
                e = cudaGraphAddNode(&node, cg, deps, edges, n_deps, &np);
                if (e == cudaSuccess) {
                    body = np.conditional.phGraph_out[0];
                    e = cudaStreamUpdateCaptureDependencies(h->stream, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
                }
            }
        }
        cudaGraph_t g_end = nullptr;
        const cudaError_t e_end = cudaStreamEndCapture(h->stream, &g_end);
        if (e == cudaSuccess) e = e_end;
        cur = body;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(out, top, 0);
    cudaGraphDestroy(top);
    CK(e);
    return LSD_OK;
}

int ensure_graphs(lsd_handle *h) {
    if (!h->g_window) TRY(h->stage_len ? build_staged_graph(h, &h->g_window) : build_graph(h, window_fn, &h->g_window));
    if (!h->g_plain) TRY(build_graph(h, enqueue_plain, &h->g_plain));
    if (h->pipe_on)
        for (int b = 0; b < 2; ++b)
            if (!h->g_round[b]) TRY(build_round_graph(h, b, &h->g_round[b]));
    return LSD_OK;
}

bool pipelined(const lsd_handle *h) { return h->pipe_on && !h->ec_on; }

// Launches n windows: one graph each, or (pipelined) one round each.
int launch_windows(lsd_handle *h, long long n) {
    if (pipelined(h)) {
        if (!h->pipe_primed) enqueue_prime(h);
        for (long long k = 0; k < n; ++k) {
            CK(cudaGraphLaunch(h->g_round[h->pipe_cur], h->stream));
            h->pipe_cur ^= 1;
        }
    } else {
        for (long long k = 0; k < n; ++k) CK(cudaGraphLaunch(h->g_window, h->stream));
    }
    return LSD_OK;
}

int read_state(lsd_handle *h, DevState *out) {
    CK(cudaMemcpyAsync(out, h->st, sizeof(DevState), cudaMemcpyDeviceToHost, h->stream));
    TRY(wait_stream(h));
    return LSD_OK;
}

__global__ void set_target_kernel(DevState *st, long long target, int relative) {
    st->target_step = relative ? st->step + target : target;
}

// The stop step is written by a one-thread kernel (the value travels as a
// kernel argument), so no host buffer has to outlive the call.
int set_target_step(lsd_handle *h, long long target, bool relative = false) {
    set_target_kernel<<<1, 1, 0, h->stream>>>(h->st, target, relative ? 1 : 0);
    CK(cudaGetLastError());
    h->unbounded = false;
    return LSD_OK;
}

int check_err(const DevState &s) {
    if (s.err & 2) return LSD_ENONFINITE;
    if (s.err & 1) return LSD_EOVERFLOW;
    if (s.err & 4) return LSD_ESTATE;
    if (s.err & (8 | 16)) return LSD_ETIMEOUT;   // a bounded device wait gave up (MLP pipeline, transport barrier)
    return LSD_OK;
}

// p <- OB(q, p_obabo) at step index n: target forces at q, then the leading
// O and B half-steps of the staggered frame (App. E).
int obabo_enter(lsd_handle *h, long long n) {
    const size_t D = 3 * (size_t)h->N;
    cudaStream_t s = h->stream;
    CK(cudaMemcpyAsync(h->p, h->p_obabo, D * sizeof(double), cudaMemcpyDeviceToDevice, s));
    launch_fixpoint(h->q, h->species, h->N, h->geo, h->fix_eval, s);
    enqueue_eval(h, h->target, h->fix_eval, 1, h->w_Ft, nullptr, s);
    launch_obabo_enter(h->geo, h->coef, h->species, h->w_Ft, n, h->p, s);
    CK(cudaGetLastError());
    TRY(wait_stream(h));
    DevState st;
    TRY(read_state(h, &st));
    return check_err(st);
}

// The activation and gradient scales of FP8 and F16x3 potentials, once per
// handle.  A calibration kernel (BF16 for FP8, the unscaled TF32 split for
// F16x3) runs the potential's MLP on the initial configuration (N rows) and
// records |max| of every A operand tensor.  FP8: the scale is 2 |max| / 448,
// so values up to twice the calibration range are represented and larger ones
// saturate; the fixed scales keep the FP8 potential one function of the
// configuration for the handle's lifetime.  F16x3: the power of two that puts
// |max| in (2^5, 2^6]; scaling is exact, so the result does not depend on it
// as long as values stay below 2^16 (1024x the calibration range).
int calibrate_scales(lsd_handle *h, PotHost &ph) {
    const PotDev &P = ph.dev;
    const int L = P.n_layers, N = h->N;
    cudaStream_t s = h->stream;
    launch_fixpoint(h->q, h->species, N, h->geo, h->fix_eval, s);
    launch_neigh_build(h->fix_eval, N, h->geo, ph.rmax2f, ph.near2f, h->cap_near, h->cap_far, h->near_keys,
                       h->far_keys, h->n_near, h->n_far, h->st, s);
    launch_desc(h->fix_eval, h->near_keys, h->n_near, h->cap_near, N, h->geo, P, h->X, s, mom_for(h, ph));
    CK(cudaMemsetAsync(ph.tc_amax, 0, 2 * L * sizeof(float), s));
    launch_mlp_tc(ph.cal_plan, h->X, N, P, h->E_mlp, h->dEdX, ph.tc_scratch, nullptr, ph.tc_amax, h->n_sm,
                  &h->st->err, s);
    CK(cudaGetLastError());
    std::vector<float> am(2 * L), sc(2 * L);
    CK(cudaMemcpyAsync(am.data(), ph.tc_amax, 2 * L * sizeof(float), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const bool f8 = mlp_tc_plan_op(ph.tc_plan) == kTcFP8;
    for (int k = 0; k < 2 * L; ++k) {
        if (!(am[k] > 0.f)) sc[k] = 1.f;
        else if (f8) sc[k] = 2.f * am[k] / 448.f;                                // e4m3: 2 |max| at the top
        else sc[k] = std::ldexp(1.f, (int)std::ceil(std::log2(am[k])) - 6);   // F16x3: |max| at 2^6, exact
    }
    CK(cudaMemcpyAsync(ph.tc_scales, sc.data(), 2 * L * sizeof(float), cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
    DevState st;
    TRY(read_state(h, &st));
    return check_err(st);
}


// The force-matching gradient of n_frames frames (slots frame0.. mod n_avail
// of fq [.][N][3] / fF) of a learned draft whose frames exceed one block:
// per frame, the frame's neighbour lists (the window's Verlet machinery, or
// all atoms without a cell grid), the draft's descriptors, the trainer's MLP
// with its pre-activations, the draft forces by the pair-gradient and gather
// kernels, then the residual, the descriptor JVP and the per-weight sums.  The
// sum over frames, and Adam when asked, follow.
int train_large_pass(lsd_handle *h, const double *fq, const float *fF, long long frame0, long long n_avail,
                     int n_frames, bool adam, float lr) {
    TrainState &t = h->train;
    TRY(train_large_bufs(t, n_frames));
    const int N = h->N;
    const PotHost &ph = h->draft;
    const PotDev &P = ph.dev;
    cudaStream_t s = h->stream;
    const float scale = -2.0f / ((float)n_frames * 3.0f * (float)N);
    const size_t D = 3 * (size_t)N;
    for (int f = 0; f < n_frames; ++f) {
        const long long slot = (frame0 + f) % n_avail;
        const double *q = fq + (size_t)slot * D;
        const float *Fs = fF + (size_t)slot * D;
        launch_fixpoint(q, h->species, N, h->geo, h->fix_eval, s);
        if (!h->vplan.all_pairs) {
            launch_verlet_build(h->vplan, q, h->species, h->geo, h->vbufs, h->st, s);
            launch_neigh_list(h->fix_eval, h->vbufs.vlist, h->vbufs.vcount, h->vplan.cap, N, h->geo, ph.rmax2f,
                              ph.near2f, h->cap_near, h->cap_far, h->near_keys, h->far_keys, h->n_near, h->n_far,
                              h->st, nullptr, s);
        } else {
            launch_neigh_build(h->fix_eval, N, h->geo, ph.rmax2f, ph.near2f, h->cap_near, h->cap_far, h->near_keys,
                               h->far_keys, h->n_near, h->n_far, h->st, s);
        }
        launch_desc(h->fix_eval, h->near_keys, h->n_near, h->cap_near, N, h->geo, P, h->X, s);
        launch_fm_mlp(t, h->X, P.d0p, h->dEdX, s);
        launch_pairgrad(h->fix_eval, h->near_keys, h->n_near, h->far_keys, h->n_far, h->cap_near, h->cap_far, N,
                        h->geo, P, h->dEdX, h->pair_g, h->Fpart, h->E_lj, s);
        launch_force_gather(h->near_keys, h->n_near, h->cap_near, N, N, 1, h->pair_g, h->Fpart, h->E_lj, h->E_mlp,
                            t.lFd, nullptr, h->st, s);
        launch_fm_frame_grad(t, h->fix_eval, h->near_keys, h->n_near, h->cap_near, h->geo, P, h->X, P.d0p, Fs, scale,
                             f, s);
    }
    launch_fm_reduce_adam(t, n_frames, adam, lr, s);
    CK(cudaGetLastError());
    h->pipe_primed = false;   // the window's Verlet lists were rebuilt for the frames
    return LSD_OK;
}

__global__ void mb_init_kernel(int N, Coef cf, const int *species, const double *mass, double T, double kT_kappa,
                               double *p) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const float3 xi = normals3(cf.seed, 0ull, (uint32_t)i, 2u);
    const double sd = sqrt(mass[species[i]] * kT_kappa);
    p[3 * i + 0] = sd * (double)xi.x;
    p[3 * i + 1] = sd * (double)xi.y;
    p[3 * i + 2] = sd * (double)xi.z;
}

}  // namespace

extern "C" {

int lsd_train_draft(lsd_handle *h, int32_t n_iters, float lr, int32_t frames_per_iter, float *loss_out);

const char *lsd_strerror(int code) {
    switch (code) {
        case LSD_OK: return "ok";
        case LSD_EINVAL: return "invalid argument";
        case LSD_ENOMEM: return "out of memory";
        case LSD_ECUDA: return g_last_cuda != cudaSuccess ? cudaGetErrorString(g_last_cuda) : "CUDA error";
        case LSD_ETIMEOUT: return "timed out waiting for the device";
        case LSD_ENONFINITE: return "non-finite force or log ratio";
        case LSD_ESTATE: return "call out of order or inconsistent neighbour lists";
        case LSD_EOVERFLOW: return "neighbour list capacity exceeded";
        case LSD_EUNSUPPORTED: return "unsupported combination of options";
        default: return "unknown error";
    }
}

void lsd_destroy(lsd_handle *h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    if (h->dstream) cudaStreamSynchronize(h->dstream);
    destroy_graphs(h);
    for (cudaEvent_t e : {h->ev_fork, h->ev_v, h->ev_d, h->ev_sync})
        if (e) cudaEventDestroy(e);
    if (h->dstream) cudaStreamDestroy(h->dstream);
    for (void *v : h->allocs) cudaFree(v);
    if (h->draft.tc_plan) mlp_tc_plan_free(h->draft.tc_plan);
    if (h->target.tc_plan) mlp_tc_plan_free(h->target.tc_plan);
    if (h->draft.cal_plan) mlp_tc_plan_free(h->draft.cal_plan);
    if (h->target.cal_plan) mlp_tc_plan_free(h->target.cal_plan);
    train_free(h->train);
    if (h->own_stream) cudaStreamDestroy(h->own_stream);
    delete h;
}

int lsd_init(const lsd_system *sys, const lsd_potential *draft, const lsd_potential *target, double gamma, double dt,
             double T, int32_t K, lsd_handle **out) {
    if (!out) return LSD_EINVAL;
    *out = nullptr;
    if (!sys || !draft || !target || !sys->pos || !sys->species || !sys->species_mass) return LSD_EINVAL;
    if (sys->n_atoms < 1 || sys->n_species < 1 || sys->n_species > kMaxSpecies) return LSD_EINVAL;
    if (K < 1 || K > kMaxK || !(dt > 0) || !(gamma >= 0) || !(T >= 0)) return LSD_EINVAL;
    for (int a = 0; a < 3; ++a)
        if (!(sys->box[a] > 0)) return LSD_EINVAL;
    for (int s = 0; s < sys->n_species; ++s)
        if (!(sys->species_mass[s] > 0)) return LSD_EINVAL;
    for (int i = 0; i < sys->n_atoms; ++i)
        if (sys->species[i] < 0 || sys->species[i] >= sys->n_species) return LSD_EINVAL;
    lsd_handle *h = new (std::nothrow) lsd_handle();
    if (!h) return LSD_ENOMEM;
    int rc = LSD_OK;
    auto fail = [&](int r) {
        lsd_destroy(h);
        return r;
    };
    if (cudaGetDevice(&h->dev) != cudaSuccess) return fail(LSD_ECUDA);
    if (cudaDeviceGetAttribute(&h->n_sm, cudaDevAttrMultiProcessorCount, h->dev) != cudaSuccess) return fail(LSD_ECUDA);
    if (cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking) != cudaSuccess) return fail(LSD_ECUDA);
    h->stream = h->own_stream;
    h->N = sys->n_atoms;
    h->S = sys->n_species;
    h->K = K;
    for (int a = 0; a < 3; ++a) h->box[a] = sys->box[a];
    h->gamma = gamma;
    h->dt = dt;
    h->T = T;
    h->seed = sys->seed;
    h->species_h.assign(sys->species, sys->species + sys->n_atoms);
    h->mass_h.assign(sys->species_mass, sys->species_mass + sys->n_species);
    Geo &g = h->geo;
    g.N = h->N;
    g.S = h->S;
    for (int a = 0; a < 3; ++a) {
        g.scale[a] = kTwo32 / h->box[a];
        g.scale_f[a] = (float)(h->box[a] / kTwo32);
        g.Lf[a] = (float)h->box[a];
    }
    // Eq. 4 coefficients
    Coef &c = h->coef;
    const double kap = kappa_conv(), kB = kboltz_ev();
    c.c1 = std::exp(-gamma * dt);
    const double hh = 0.5 * dt;
    c.aF = (1.0 + c.c1) * hh * kap;
    const double one_minus = -std::expm1(-2.0 * gamma * dt);
    for (int s = 0; s < h->S; ++s) {
        const double m = h->mass_h[s];
        c.hm[s] = hh / m;
        c.sig[s] = std::sqrt(m * kB * T * kap * one_minus);
        c.aF_sig[s] = c.sig[s] > 0 ? c.aF / c.sig[s] : 0.0;
    }
    c.seed = h->seed;
    // App. E: the staggered OBABO frame (used after lsd_set_integrator(h, LSD_OBABO))
    c.obabo = 0;
    c.ch = std::exp(-0.5 * gamma * dt);
    c.bF = hh * kap;
    c.ob_a = c.ch / (1.0 + c.c1);
    c.ob_b = std::sqrt(1.0 / (1.0 + c.c1));
    const double one_minus_half = -std::expm1(-gamma * dt);
    for (int s = 0; s < h->S; ++s) {
        const double m = h->mass_h[s];
        c.hmf[s] = dt / m;
        c.sigh[s] = std::sqrt(m * kB * T * kap * one_minus_half);
    }
    if ((rc = pot_setup(h, h->draft, draft, true)) != LSD_OK) return fail(rc);
    if ((rc = pot_setup(h, h->target, target, false)) != LSD_OK) return fail(rc);
    h->learned_small = h->draft.dev.has_mlp;
    if (mlp_fp32_smem_bytes(h->target.dev) > (size_t)kMaxDynSmem) return fail(LSD_EUNSUPPORTED);
    // capacities from the mean density (x2 + margin)
    const double V = h->box[0] * h->box[1] * h->box[2];
    const double rho = h->N / V;
    double rnear = 0.0, rfar = 0.0;
    for (const PotHost *ph : {&h->draft, &h->target}) {
        rnear = std::max(rnear, ph->dev.has_mlp ? (double)ph->p.desc_cutoff : 0.0);
        rfar = std::max(rfar, std::max(ph->dev.has_lj ? ph->p.lj_cutoff : 0.0, ph->dev.has_mlp ? ph->p.desc_cutoff : 0.0));
    }
    h->cap_near = std::min(nb_capacity(rho, rnear, 32), (27 * h->N + 31) / 32 * 32);
    h->cap_far = std::min(nb_capacity(rho, rfar, 32), (27 * h->N + 31) / 32 * 32);
    if (h->learned_small) {
        const double rcd = std::max(h->draft.dev.has_lj ? h->draft.p.lj_cutoff : 0.0, h->draft.p.desc_cutoff);
        h->nbr_cap = std::min(nb_capacity(rho, rcd, 32), (27 * h->N + 31) / 32 * 32);
    }
    // the target's angular block by moments when rows hold many neighbours: 165 monomials per neighbour instead
    // of n / 2 pair terms pay from about 40 neighbours on
    if (h->target.dev.has_mlp && h->target.dev.n_ang) {
        const double rd = h->target.p.desc_cutoff;
        h->mom_on = rho * 4.0 / 3.0 * M_PI * rd * rd * rd >= kMomMinNeighbours;
    }
    // the pair-gradient kernel: staging, dE/dX and the q-side hand-over buffer per warp; at most 16 neighbours per lane
    if (h->cap_near > 512 ||
        desc_smem_bytes(8, h->cap_near) + 8 * (256 + 4 * h->cap_near) * sizeof(float) > (size_t)kMaxDynSmem)
        return fail(LSD_EUNSUPPORTED);
    if (verify_kernels_setup(kMaxDynSmem) != cudaSuccess || mlp_kernels_setup(kMaxDynSmem) != cudaSuccess ||
        mlp_tc_setup() != cudaSuccess ||
        draft_kernels_setup(kMaxDynSmem) != cudaSuccess || transport_setup() != cudaSuccess ||
        verlet_setup(kMaxDynSmem) != cudaSuccess)
        return fail(LSD_ECUDA);
    {
        // Verlet lists: skin from the lightest species' thermal speed over a window (1 to 2.5 A)
        double mmin = h->mass_h[0];
        for (double m : h->mass_h) mmin = std::min(mmin, m);
        const double v1 = std::sqrt(kB * T * kap / mmin);
        const double skin = std::min(2.5, std::max(1.0, 5.0 * v1 * K * dt));
        const double rlist = rfar + skin;
        h->list_rcut = rfar;
        h->list_skin0 = h->list_skin = skin;
        VerletPlan &vp = h->vplan;
        for (int a = 0; a < 3; ++a) vp.nc[a] = std::max(1, (int)std::floor(h->box[a] / rlist));
        vp.all_pairs = vp.nc[0] < 3 || vp.nc[1] < 3 || vp.nc[2] < 3;
        vp.rlist2f = (float)(rlist * rlist);
        vp.move2f = (float)((0.45 * skin) * (0.45 * skin));
        h->move2f_list = vp.move2f;
        vp.cap = std::min(nb_capacity(rho, rlist, 32), (h->N + 31) / 32 * 32);
        vp.cap_pow2 = 32;
        while (vp.cap_pow2 < vp.cap) vp.cap_pow2 *= 2;
        if ((size_t)8 * vp.cap_pow2 * sizeof(int) > (size_t)kMaxDynSmem) return fail(LSD_EUNSUPPORTED);
        // the largest cluster the hardware co-schedules with the plan's shared memory
        h->dplan = draft_plan(h->N, K, h->draft.dev, h->learned_small, vp.cap, vp.all_pairs, 16, kMaxDynSmem);
        const int maxc = draft_max_cluster(h->dplan.smem, h->learned_small);
        if (maxc < h->dplan.cluster)
            h->dplan = draft_plan(h->N, K, h->draft.dev, h->learned_small, vp.cap, vp.all_pairs, maxc, kMaxDynSmem);
        {
            double rcd = h->draft.p.lj_cutoff;
            if (h->learned_small) rcd = std::max(rcd, h->draft.p.desc_cutoff);
            const double lmin = std::min(h->box[0], std::min(h->box[1], h->box[2]));
            h->dplan.minimg = rcd < 0.499 * lmin;
        }
        if (!h->dplan.ok) return fail(LSD_EUNSUPPORTED);
        // large systems: the grid form for every draft that has the GPU to itself
        if (h->N >= kGridDraftMinAtoms) {
            DraftPlan gp = draft_grid_plan(h->N, K, h->draft.dev, h->learned_small, vp.cap, vp.all_pairs, h->n_sm,
                                           kMaxDynSmem);
            gp.minimg = h->dplan.minimg;
            if (gp.ok && draft_grid_fits(gp, h->learned_small, h->n_sm)) {
                h->gplan = gp;
                h->grid_draft = true;
            }
            cudaGetLastError();
        }
        h->dplan0 = h->dplan;
        h->gplan0 = h->gplan;
        // programmatic dependent launches pay in launch-bound windows and cost about a tenth of the window
        // where kernels fill the GPU (4,096 and 32,768 atoms, measured)
        h->pdl_graphs = h->N < kGridDraftMinAtoms;
    }
    const size_t N = h->N, D = 3 * N, KN = (size_t)K * N, KD = (size_t)K * D;
    const int dmax = std::max(h->draft.dev.d0p, h->target.dev.d0p);
    // q and p in one allocation, p right after q: a host state laid out the same way moves in one copy
    if ((rc = dalloc(h, &h->q, 2 * D)) || (rc = dalloc(h, &h->p_obabo, D)) || (rc = dalloc(h, &h->species, N)) ||
        (rc = dalloc(h, &h->st, 1)) || (rc = dalloc(h, &h->w_qmid, KD)) || (rc = dalloc(h, &h->w_pdraft, KD)) ||
        (rc = dalloc(h, &h->w_Fd, KD)) || (rc = dalloc(h, &h->w_Fraw, KD)) || (rc = dalloc(h, &h->w_Ft, KD)) ||
        (rc = dalloc(h, &h->w_fix, KN)) || (rc = dalloc(h, &h->fix_eval, KN)) || (rc = dalloc(h, &h->ec_dF, D)) ||
        (rc = dalloc(h, &h->near_keys, KN * h->cap_near)) || (rc = dalloc(h, &h->far_keys, KN * h->cap_far)) ||
        (rc = dalloc(h, &h->n_near, KN)) || (rc = dalloc(h, &h->n_far, KN)) ||
        (rc = dalloc(h, &h->X, KN * std::max(dmax, 32))) || (rc = dalloc(h, &h->dEdX, KN * std::max(dmax, 32))) ||
        (rc = dalloc(h, &h->E_mlp, KN)) || (rc = dalloc(h, &h->E_lj, KN)) || (rc = dalloc(h, &h->E_atom, KN)) ||
        (rc = dalloc(h, &h->pair_g, KN * h->cap_near)) || (rc = dalloc(h, &h->Fpart, KN)) ||
        (rc = dalloc(h, &h->partials, (size_t)K * ((h->N + 1023) / 1024 + 600))) ||
        (rc = dalloc(h, &h->w_dEdX, N * std::max(h->draft.dev.d0p, 32))) ||
        (rc = dalloc(h, &h->w_nbr, h->learned_small ? N * ((size_t)h->nbr_cap + 1) : 1)) ||
        (rc = dalloc(h, &h->dsync, 1)) || (rc = dalloc(h, &h->mom, h->mom_on ? KN * kMomRowFloats : 1)) ||
        (rc = dalloc(h, &h->vbufs.fix_base, N)) || (rc = dalloc(h, &h->vbufs.cell_of_atom, N)) ||
        (rc = dalloc(h, &h->vbufs.cell_count, (size_t)h->vplan.nc[0] * h->vplan.nc[1] * h->vplan.nc[2])) ||
        (rc = dalloc(h, &h->vbufs.cell_start, (size_t)h->vplan.nc[0] * h->vplan.nc[1] * h->vplan.nc[2] + 1)) ||
        (rc = dalloc(h, &h->vbufs.cell_atoms, N)) || (rc = dalloc(h, &h->vbufs.cell_scratch, 1)) ||
        (rc = dalloc(h, &h->vbufs.vlist, N * h->vplan.cap)) || (rc = dalloc(h, &h->vbufs.vcount, N)))
        return fail(rc);
    h->p = h->q + D;
    h->wb[0].qmid = h->w_qmid;
    h->wb[0].pdraft = h->w_pdraft;
    h->wb[0].Fd = h->w_Fd;
    h->wb[0].Fraw = h->w_Fraw;
    h->wb[0].fix = h->w_fix;
    h->wb[0].vb = h->vbufs;
    if ((rc = pot_upload(h, h->draft)) != LSD_OK) return fail(rc);
    if ((rc = pot_upload(h, h->target)) != LSD_OK) return fail(rc);
    // MLPs on the tensor cores: BF16 as is, FP32 as three TF32 products, FP8 e4m3
    for (PotHost *ph : {&h->draft, &h->target}) {
        const PotDev &P = ph->dev;
        if (!P.has_mlp) continue;
        int op = -1;
        if (P.precision == LSD_BF16) op = kTcBF16;
        if (P.precision == LSD_FP32_TF32 && mlp_tc_supported(kTcTF32x3, P)) op = kTcTF32x3;
        if (P.precision == LSD_FP32 && mlp_tc_supported(kTcF16x3, P)) op = kTcF16x3;
        if (P.precision == LSD_FP8) op = kTcFP8;
        if (op < 0) continue;   // FP32 beyond the split kernels' shapes, or LSD_FP32_CUDA_CORES: CUDA cores
        if (!mlp_tc_supported(op, P)) return fail(LSD_EUNSUPPORTED);
        TcWeights w{}, wb{}, wtf{};
        for (int l = 0; l < P.n_layers; ++l) {
            const size_t on = P.Wn[l] - ph->dbuf, ot = P.Wt[l] - ph->dbuf;
            wb.wn[l][0] = P.Wn_bf[l];
            wb.wt[l][0] = P.Wt_bf[l];
            if (ph->dbuf_tf) {
                wtf.wn[l][0] = ph->dbuf_tf + on;
                wtf.wn[l][1] = ph->dbuf_tf + ph->n_dbuf + on;
                wtf.wt[l][0] = ph->dbuf_tf + ot;
                wtf.wt[l][1] = ph->dbuf_tf + ph->n_dbuf + ot;
            }
            if (op == kTcF16x3) {
                w.wn[l][0] = ph->dbuf_h + on;
                w.wn[l][1] = ph->dbuf_h + ph->n_dbuf + on;
                w.wt[l][0] = ph->dbuf_h + ot;
                w.wt[l][1] = ph->dbuf_h + ph->n_dbuf + ot;
            } else if (op == kTcTF32x3) {
                w.wn[l][0] = ph->dbuf_tf + on;
                w.wn[l][1] = ph->dbuf_tf + ph->n_dbuf + on;
                w.wt[l][0] = ph->dbuf_tf + ot;
                w.wt[l][1] = ph->dbuf_tf + ph->n_dbuf + ot;
            } else if (op == kTcFP8) {
                w.wn[l][0] = ph->dbuf_f8 + on;
                w.wt[l][0] = ph->dbuf_f8 + ot;
            } else {
                w = wb;
            }
        }
        ph->tc_plan = mlp_tc_plan(op, P, w);
        if (!ph->tc_plan) return fail(LSD_ECUDA);
        if (op == kTcFP8 || op == kTcF16x3) {
            // the calibration run: BF16 for FP8, the unscaled TF32 split for F16x3
            ph->cal_plan = op == kTcFP8 ? mlp_tc_plan(kTcBF16, P, wb) : mlp_tc_plan(kTcTF32x3, P, wtf);
            if (!ph->cal_plan) return fail(LSD_ECUDA);
        }
        const int grid = mlp_tc_grid(h->K * h->N, h->n_sm);
        const size_t ns = mlp_tc_scratch_elems(op, P, grid);
        if (ns && (rc = dalloc(h, &ph->tc_scratch, ns)) != LSD_OK) return fail(rc);
    }
    if (cudaMemcpy(h->q, sys->pos, D * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(h->species, sys->species, N * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(LSD_ECUDA);
    DevState s0{};
    s0.step = 0;
    s0.target_step = 0;
    s0.first_reject_last = -1;
    s0.spec_ema = 1.f;
    s0.list_force = 1;   // no lists yet
    if (cudaMemcpy(h->st, &s0, sizeof(DevState), cudaMemcpyHostToDevice) != cudaSuccess) return fail(LSD_ECUDA);
    if (sys->mom) {
        if (cudaMemcpy(h->p, sys->mom, D * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
            return fail(LSD_ECUDA);
    } else {
        double *dmass = nullptr;
        if ((rc = dalloc(h, &dmass, h->S)) != LSD_OK) return fail(rc);
        if (cudaMemcpy(dmass, h->mass_h.data(), h->S * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
            return fail(LSD_ECUDA);
        mb_init_kernel<<<(h->N + 255) / 256, 256, 0, h->stream>>>(h->N, h->coef, h->species, dmass, T, kB * T * kap,
                                                                  h->p);
        if (cudaStreamSynchronize(h->stream) != cudaSuccess) return fail(LSD_ECUDA);
    }
    if ((rc = train_init(h->train, h->draft.dev, h->draft.weights, h->N)) != LSD_OK) return fail(rc);
    h->train.st = h->st;
    h->train.K = K;
    {
        // plain target steps in one fused cooperative launch when the system is small and the target's network FP32
        const int tp = h->target.p.precision;
        const bool fp32 = tp == LSD_FP32 || tp == LSD_FP32_TF32 || tp == LSD_FP32_CUDA_CORES;
        h->pplan = plain_plan(h->N, h->target.dev, fp32, false, h->cap_near, h->geo, kMaxDynSmem);
        if (h->pplan.ok && plain_setup(h->pplan) != cudaSuccess) h->pplan.ok = false;
        cudaGetLastError();   // a configuration the device cannot co-schedule only disables the fused step
        if (h->pplan.ok) {
            if ((rc = dalloc(h, &h->pf_fix, N)) || (rc = dalloc(h, &h->pf_keys, N * h->pplan.cap)) ||
                (rc = dalloc(h, &h->pf_cnt, N)) || (rc = dalloc(h, &h->pf_pg, N * h->pplan.cap)) ||
                (rc = dalloc(h, &h->pf_bar, 1)))
                return fail(rc);
            h->plain_fused = true;
        }
    }
    for (PotHost *ph : {&h->draft, &h->target})
        if (ph->cal_plan && (rc = calibrate_scales(h, *ph)) != LSD_OK) return fail(rc);
    if (cudaDeviceSynchronize() != cudaSuccess) return fail(LSD_ECUDA);
    *out = h;
    return LSD_OK;
}

int lsd_set_stream(lsd_handle *h, void *cuda_stream) {
    if (!h) return LSD_EINVAL;
    CK(cudaStreamSynchronize(h->stream));
    h->stream = cuda_stream ? (cudaStream_t)cuda_stream : h->own_stream;
    destroy_graphs(h);
    return LSD_OK;
}

int lsd_draft_window(lsd_handle *h) {
    if (!h) return LSD_EINVAL;
    DevState s;
    TRY(read_state(h, &s));
    TRY(set_target_step(h, s.step + h->K));
    h->pipe_primed = false;   // the per-window calls use window buffer 0
    enqueue_draft(h, h->stream);
    CK(cudaGetLastError());
    h->drafted = true;
    return LSD_OK;
}

int lsd_verify_window(lsd_handle *h, int32_t *n_committed, int32_t *first_reject) {
    if (!h) return LSD_EINVAL;
    if (!h->drafted) return LSD_ESTATE;
    enqueue_verify(h, h->stream);
    CK(cudaGetLastError());
    h->drafted = false;
    DevState s;
    TRY(read_state(h, &s));
    if (n_committed) *n_committed = s.n_commit_last;
    if (first_reject) *first_reject = s.first_reject_last;
    return check_err(s);
}

int lsd_transport_window(lsd_handle *h, const double *q_mid, const double *p_draft, const float *F_draft,
                         const float *F_target, int32_t k, int32_t *n_committed, int32_t *first_reject) {
    if (!h || !q_mid || !p_draft || !F_draft || !F_target || k < 1 || k > h->K) return LSD_EINVAL;
    TRY(wait_stream(h));
    const size_t bytes_d = (size_t)k * 3 * h->N * sizeof(double), bytes_f = (size_t)k * 3 * h->N * sizeof(float);
    cudaStream_t s = h->stream;
    CK(cudaMemcpyAsync(h->w_qmid, q_mid, bytes_d, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(h->w_pdraft, p_draft, bytes_d, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(h->w_Fd, F_draft, bytes_f, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(h->w_Fraw, F_draft, bytes_f, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(h->w_Ft, F_target, bytes_f, cudaMemcpyHostToDevice, s));
    const int keff = k;
    CK(cudaMemcpyAsync(&h->st->k_eff, &keff, sizeof(int), cudaMemcpyHostToDevice, s));
    DevState st;
    TRY(read_state(h, &st));
    TRY(set_target_step(h, st.step + k));
    h->drafted = false;
    h->pipe_primed = false;   // window buffer 0 now holds the given window
    launch_transport(h->K, h->geo, h->coef, h->species, h->w_qmid, h->w_pdraft, h->w_Fd, h->w_Ft, h->w_Fraw,
                     h->ec_dF, h->ec_on, h->q, h->p, h->p_obabo, h->st, h->partials, &h->st->k_eff, s);
    CK(cudaGetLastError());
    TRY(read_state(h, &st));
    if (n_committed) *n_committed = st.n_commit_last;
    if (first_reject) *first_reject = st.first_reject_last;
    return check_err(st);
}

int lsd_step(lsd_handle *h, int64_t n_steps, lsd_stats *stats) {
    if (!h || n_steps < 0) return LSD_EINVAL;
    TRY(ensure_graphs(h));
    DevState s;
    TRY(read_state(h, &s));
    const long long target = s.step + n_steps;
    TRY(set_target_step(h, target));
    long long w0 = s.windows, c0 = s.committed;
    long long rem = n_steps;
    while (rem > 0) {
        double rate = (s.windows > w0) ? (double)(s.committed - c0) / (double)(s.windows - w0) : (double)h->K;
        if (rate < 1.0) rate = 1.0;
        long long batch = (long long)std::ceil((double)rem / rate);
        if (h->online_every > 0) {
            // stop the batch near the next retraining point
            const long long left = h->online_every - ((s.committed - s.rejected) - h->online_base);
            const long long b2 = (long long)std::ceil((double)std::max(left, 1ll) / rate);
            batch = std::min(batch, b2);
        }
        if (batch < 1) batch = 1;
        TRY(launch_windows(h, batch));
        TRY(read_state(h, &s));
        TRY(check_err(s));
        rem = target - s.step;
        if (h->online_every > 0 && (s.committed - s.rejected) - h->online_base >= h->online_every) {
            // retrain the learned draft on the captured target-verified frames, between windows
            float loss = 0.f;
            TRY(lsd_train_draft(h, h->online_iters, h->online_lr, h->online_fpi, &loss));
            h->online_loss = loss;
            h->online_count += 1;
            h->online_base = s.committed - s.rejected;
            TRY(ensure_graphs(h));
        }
    }
    h->drafted = false;
    if (stats) TRY(lsd_get_stats(h, stats));
    return LSD_OK;
}

int lsd_enqueue_windows(lsd_handle *h, int32_t n) {
    if (!h || n < 0) return LSD_EINVAL;
    TRY(ensure_graphs(h));
    if (!h->unbounded) {
        TRY(set_target_step(h, (long long)1 << 60));
        h->unbounded = true;
    }
    TRY(launch_windows(h, n));
    h->drafted = false;
    return LSD_OK;
}

int lsd_enqueue_plain(lsd_handle *h, int32_t n) {
    if (!h || n < 0) return LSD_EINVAL;
    TRY(ensure_graphs(h));
    if (!h->unbounded) {
        TRY(set_target_step(h, (long long)1 << 60));
        h->unbounded = true;
    }
    h->pipe_primed = false;   // plain steps reuse window buffer 0
    if (use_plain_fused(h)) return launch_plain_steps_fused(h, n);
    for (int32_t k = 0; k < n; ++k) CK(cudaGraphLaunch(h->g_plain, h->stream));
    return LSD_OK;
}

int lsd_plain_step(lsd_handle *h, int64_t n_steps) {
    if (!h || n_steps < 0) return LSD_EINVAL;
    TRY(ensure_graphs(h));
    DevState s;
    TRY(read_state(h, &s));
    TRY(set_target_step(h, s.step + n_steps));
    h->pipe_primed = false;   // plain steps reuse window buffer 0
    if (use_plain_fused(h)) {
        TRY(launch_plain_steps_fused(h, n_steps));
    } else {
        for (int64_t t = 0; t < n_steps; ++t) CK(cudaGraphLaunch(h->g_plain, h->stream));
    }
    TRY(read_state(h, &s));
    return check_err(s);
}

int lsd_get_stats(const lsd_handle *h, lsd_stats *out) {
    if (!h || !out) return LSD_EINVAL;
    DevState s;
    TRY(read_state(const_cast<lsd_handle *>(h), &s));
    out->windows = s.windows;
    out->committed = s.committed;
    out->rejected = s.rejected;
    out->verified = s.verified;
    out->sum_delta = s.sum_delta;
    out->sum_pred_reject = s.sum_pred;
    out->step = s.step;
    out->stages = s.stages;
    out->list_builds = s.list_builds;
    return LSD_OK;
}

int lsd_window_host(lsd_handle *h, const double *pos, const double *mom, int64_t step, double *pos_out,
                    double *mom_out, int64_t *step_out, int32_t *n_committed) {
    if (!h || !pos || !mom || !pos_out || !mom_out || step < 0) return LSD_EINVAL;
    TRY(ensure_graphs(h));
    const size_t D = 3 * (size_t)h->N;
    double *pm = h->coef.obabo ? h->p_obabo : h->p;
    if (pm == h->q + D && mom == pos + D) {   // [pos; mom] adjacent on both sides
        CK(cudaMemcpyAsync(h->q, pos, 2 * D * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    } else {
        CK(cudaMemcpyAsync(h->q, pos, D * sizeof(double), cudaMemcpyHostToDevice, h->stream));
        CK(cudaMemcpyAsync(pm, mom, D * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    }
    // step and stop step of the run state, adjacent: one copy
    static_assert(offsetof(DevState, target_step) == offsetof(DevState, step) + sizeof(long long), "layout");
    long long head[2] = {step, step + h->K};
    CK(cudaMemcpyAsync(&h->st->step, head, sizeof(head), cudaMemcpyHostToDevice, h->stream));
    h->unbounded = false;
    h->drafted = false;
    h->pipe_primed = false;
    if (h->coef.obabo) TRY(obabo_enter(h, step));
    CK(cudaGraphLaunch(h->g_window, h->stream));
    if (pm == h->q + D && mom_out == pos_out + D) {
        CK(cudaMemcpyAsync(pos_out, h->q, 2 * D * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    } else {
        CK(cudaMemcpyAsync(pos_out, h->q, D * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        CK(cudaMemcpyAsync(mom_out, pm, D * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    }
    // step, stop step, committed count, first rejection, k_eff, error flags: the first 32 bytes
    struct Head {
        long long step, target;
        int n_commit, first_reject, k_eff, err;
    } out{};
    static_assert(offsetof(DevState, err) + sizeof(int) == sizeof(Head), "layout");
    CK(cudaMemcpyAsync(&out, h->st, sizeof(Head), cudaMemcpyDeviceToHost, h->stream));
    TRY(wait_stream(h));
    if (step_out) *step_out = out.step;
    if (n_committed) *n_committed = out.n_commit;
    DevState s{};
    s.err = out.err;
    return check_err(s);
}

int lsd_get_state(const lsd_handle *hc, double *pos, double *mom, int64_t *step) {
    if (!hc) return LSD_EINVAL;
    lsd_handle *h = const_cast<lsd_handle *>(hc);
    const size_t D = 3 * (size_t)h->N;
    if (pos) CK(cudaMemcpyAsync(pos, h->q, D * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    const double *pm = h->coef.obabo ? h->p_obabo : h->p;   // OBABO: the recovered output momentum
    if (mom) CK(cudaMemcpyAsync(mom, pm, D * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    long long st = 0;
    CK(cudaMemcpyAsync(&st, &h->st->step, sizeof(long long), cudaMemcpyDeviceToHost, h->stream));
    TRY(wait_stream(h));
    if (step) *step = st;
    return LSD_OK;
}

int lsd_set_state(lsd_handle *h, const double *pos, const double *mom, int64_t step) {
    if (!h || step < 0) return LSD_EINVAL;
    const size_t D = 3 * (size_t)h->N;
    if (pos) CK(cudaMemcpyAsync(h->q, pos, D * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    if (mom) CK(cudaMemcpyAsync(h->coef.obabo ? h->p_obabo : h->p, mom, D * sizeof(double), cudaMemcpyHostToDevice,
                                h->stream));
    long long st = step;
    CK(cudaMemcpyAsync(&h->st->step, &st, sizeof(long long), cudaMemcpyHostToDevice, h->stream));
    TRY(wait_stream(h));
    h->drafted = false;
    h->pipe_primed = false;
    if (h->coef.obabo) TRY(obabo_enter(h, step));   // the staggered momentum of the given OBABO state
    return LSD_OK;
}

int lsd_set_pipelining(lsd_handle *h, int32_t on) {
    if (!h) return LSD_EINVAL;
    if (on && h->ec_on) return LSD_ESTATE;   // the speculative draft would read the cache while it is rewritten
    if (on && h->stage_len) return LSD_ESTATE;   // staged windows end on the device; a round drafts past them
    if (on && h->list_reuse) return LSD_ESTATE;  // a round always builds the lists of the window it drafts
    TRY(wait_stream(h));
    if (on && !h->pipe_alloc) {
        const size_t N = h->N, D = 3 * N, KN = (size_t)h->K * N, KD = (size_t)h->K * D;
        const size_t ncell = (size_t)h->vplan.nc[0] * h->vplan.nc[1] * h->vplan.nc[2];
        lsd_handle::WinBufs &w = h->wb[1];
        int rc = LSD_OK;
        if ((rc = dalloc(h, &w.qmid, KD)) || (rc = dalloc(h, &w.pdraft, KD)) || (rc = dalloc(h, &w.Fd, KD)) ||
            (rc = dalloc(h, &w.Fraw, KD)) || (rc = dalloc(h, &w.fix, KN)) || (rc = dalloc(h, &w.vb.fix_base, N)) ||
            (rc = dalloc(h, &w.vb.cell_of_atom, N)) || (rc = dalloc(h, &w.vb.cell_count, ncell)) ||
            (rc = dalloc(h, &w.vb.cell_start, ncell + 1)) || (rc = dalloc(h, &w.vb.cell_atoms, N)) ||
            (rc = dalloc(h, &w.vb.cell_scratch, 1)) || (rc = dalloc(h, &w.vb.vlist, N * h->vplan.cap)) ||
            (rc = dalloc(h, &w.vb.vcount, N)) || (rc = dalloc(h, &h->hdr, 2)) || (rc = dalloc(h, &h->qb, D)) ||
            (rc = dalloc(h, &h->pb, D)))
            return rc;
        int lo = 0, hi = 0;
        CK(cudaDeviceGetStreamPriorityRange(&lo, &hi));
        CK(cudaStreamCreateWithPriority(&h->dstream, cudaStreamNonBlocking, hi));   // the draft is the serial chain
        CK(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&h->ev_v, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&h->ev_d, cudaEventDisableTiming));
        h->pipe_alloc = true;
    }
    h->pipe_on = on != 0;
    destroy_graphs(h);
    return LSD_OK;
}

int lsd_set_integrator(lsd_handle *h, int32_t scheme) {
    if (!h || (scheme != LSD_ABOBA && scheme != LSD_OBABO)) return LSD_EINVAL;
    const int want = scheme == LSD_OBABO ? 1 : 0;
    if (want == h->coef.obabo) return LSD_OK;
    const size_t D = 3 * (size_t)h->N;
    DevState s;
    TRY(read_state(h, &s));
    destroy_graphs(h);   // the kernels take the coefficients by value at capture
    h->drafted = false;
    if (want) {
        // the current state is an OBABO state y; the chain continues from OB(y)
        CK(cudaMemcpyAsync(h->p_obabo, h->p, D * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
        h->coef.obabo = 1;
        TRY(obabo_enter(h, s.step));
    } else {
        // the current OBABO output state becomes the ABOBA state
        CK(cudaMemcpyAsync(h->p, h->p_obabo, D * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
        h->coef.obabo = 0;
        TRY(wait_stream(h));
    }
    return LSD_OK;
}

int lsd_set_max_displacement(lsd_handle *h, double d_max) {
    if (!h || !(d_max >= 0.0)) return LSD_EINVAL;
    if (h->vplan.all_pairs && !h->dplan.self_list) return LSD_EUNSUPPORTED;   // no lists: no displacement check
    TRY(wait_stream(h));
    h->move2f_user = d_max == 0.0 ? 0.f : (float)(d_max * d_max);
    h->vplan.move2f = h->move2f_user > 0.f ? std::min(h->move2f_user, h->move2f_list) : h->move2f_list;
    destroy_graphs(h);   // the bound is a launch argument of the draft
    return LSD_OK;
}

int lsd_set_list_skin(lsd_handle *h, double skin) {
    if (!h || !(skin > 0.0) || skin > h->list_skin0) return LSD_EINVAL;
    if (h->vplan.all_pairs) return LSD_EUNSUPPORTED;   // no cell-grid lists
    TRY(wait_stream(h));
    const double rlist = h->list_rcut + skin;
    h->list_skin = skin;
    h->vplan.rlist2f = (float)(rlist * rlist);
    h->move2f_list = (float)((0.45 * skin) * (0.45 * skin));
    h->vplan.move2f = h->move2f_user > 0.f ? std::min(h->move2f_user, h->move2f_list) : h->move2f_list;
    destroy_graphs(h);   // the list radius and the bound are launch arguments
    return LSD_OK;
}

int lsd_get_list_skin(const lsd_handle *h, double *skin) {
    if (!h || !skin) return LSD_EINVAL;
    *skin = h->vplan.all_pairs ? 0.0 : h->list_skin;
    return LSD_OK;
}

int lsd_set_error_correction(lsd_handle *h, int32_t on) {
    if (!h) return LSD_EINVAL;
    if (on && h->pipe_on) return LSD_ESTATE;   // see lsd_set_pipelining
    CK(cudaMemsetAsync(h->ec_dF, 0, 3 * (size_t)h->N * sizeof(float), h->stream));
    h->ec_on = on ? 1 : 0;
    destroy_graphs(h);
    return wait_stream(h);
}

int lsd_set_draft_weights(lsd_handle *h, const float *w, size_t n) {
    if (!h || !w) return LSD_EINVAL;
    if (!h->draft.dev.has_mlp || n != h->draft.weights.size()) return LSD_EINVAL;
    TRY(wait_stream(h));
    h->draft.weights.assign(w, w + n);
    TRY(pot_upload(h, h->draft));
    TRY(train_set_weights(h->train, h->draft.weights));
    destroy_graphs(h);   // bout is a kernel parameter
    return LSD_OK;
}

int lsd_get_draft_weights(const lsd_handle *h, float *w, size_t n) {
    if (!h || !w) return LSD_EINVAL;
    if (n != h->draft.weights.size()) return LSD_EINVAL;
    std::memcpy(w, h->draft.weights.data(), n * sizeof(float));
    return LSD_OK;
}

static int forces_dev(lsd_handle *h, PotHost &pot, const double *q_dev, int32_t C, float *F_dev, float *E_dev) {
    if (!h || !q_dev || !F_dev || C < 1 || C > h->K) return LSD_EINVAL;
    const int M = C * h->N;
    launch_fixpoint(q_dev, h->species, M, h->geo, h->fix_eval, h->stream);
    enqueue_eval(h, pot, h->fix_eval, C, F_dev, E_dev, h->stream);
    CK(cudaGetLastError());
    DevState s;
    TRY(read_state(h, &s));
    return check_err(s);
}

int lsd_target_forces_dev(lsd_handle *h, const double *q_dev, int32_t C, float *F_dev, float *E_dev) {
    if (!h) return LSD_EINVAL;
    return forces_dev(h, h->target, q_dev, C, F_dev, E_dev);
}

int lsd_draft_forces_dev(lsd_handle *h, const double *q_dev, int32_t C, float *F_dev, float *E_dev) {
    if (!h) return LSD_EINVAL;
    return forces_dev(h, h->draft, q_dev, C, F_dev, E_dev);
}

int lsd_neighbors(const lsd_handle *hc, int32_t config, int32_t cap, int32_t *desc_keys, int32_t *desc_counts,
                  int32_t *lj_keys, int32_t *lj_counts) {
    if (!hc || config < 0 || config >= hc->K || cap < 1) return LSD_EINVAL;
    lsd_handle *h = const_cast<lsd_handle *>(hc);
    const size_t N = h->N, r0 = (size_t)config * N;
    std::vector<int> nk(N * h->cap_near), fk(N * h->cap_far), nn(N), nf(N);
    CK(cudaMemcpyAsync(nk.data(), h->near_keys + r0 * h->cap_near, nk.size() * sizeof(int), cudaMemcpyDeviceToHost,
                       h->stream));
    CK(cudaMemcpyAsync(fk.data(), h->far_keys + r0 * h->cap_far, fk.size() * sizeof(int), cudaMemcpyDeviceToHost,
                       h->stream));
    CK(cudaMemcpyAsync(nn.data(), h->n_near + r0, N * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(nf.data(), h->n_far + r0, N * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    TRY(wait_stream(h));
    for (size_t i = 0; i < N; ++i) {
        const int *a = nk.data() + i * h->cap_near;
        const int *b = fk.data() + i * h->cap_far;
        if (desc_keys && desc_counts) {
            if (nn[i] > cap) return LSD_EOVERFLOW;
            std::memcpy(desc_keys + i * cap, a, nn[i] * sizeof(int));
            desc_counts[i] = nn[i];
        }
        if (lj_keys && lj_counts) {
            // the LJ cutoff is the outer cutoff here: near and far lists together, merged in key order
            if (nn[i] + nf[i] > cap) return LSD_EOVERFLOW;
            std::merge(a, a + nn[i], b, b + nf[i], lj_keys + i * cap);
            lj_counts[i] = nn[i] + nf[i];
        }
    }
    return LSD_OK;
}

int lsd_descriptors(const lsd_handle *hc, int32_t C, float *X, float *dEdX) {
    if (!hc || C < 1 || C > hc->K) return LSD_EINVAL;
    lsd_handle *h = const_cast<lsd_handle *>(hc);
    const PotDev &P = h->target.dev;
    if (!P.has_mlp) return LSD_EINVAL;
    const size_t M = (size_t)C * h->N;
    std::vector<float> x(M * P.d0p), gx(M * P.d0p);
    CK(cudaMemcpyAsync(x.data(), h->X, x.size() * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(gx.data(), h->dEdX, gx.size() * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    TRY(wait_stream(h));
    for (size_t r = 0; r < M; ++r) {
        if (X) std::memcpy(X + r * P.d0, x.data() + r * P.d0p, P.d0 * sizeof(float));
        if (dEdX) std::memcpy(dEdX + r * P.d0, gx.data() + r * P.d0p, P.d0 * sizeof(float));
    }
    return LSD_OK;
}

int lsd_get_window(const lsd_handle *hc, double *q_mid, double *p_draft, float *F_draft, float *F_target,
                   double *log_ratio, double *log_u, double *delta_norm, int32_t *accept) {
    if (!hc) return LSD_EINVAL;
    lsd_handle *h = const_cast<lsd_handle *>(hc);
    const size_t KD = (size_t)h->K * 3 * h->N;
    if (q_mid) CK(cudaMemcpyAsync(q_mid, h->w_qmid, KD * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    if (p_draft) CK(cudaMemcpyAsync(p_draft, h->w_pdraft, KD * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    if (F_draft) CK(cudaMemcpyAsync(F_draft, h->w_Fd, KD * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    if (F_target) CK(cudaMemcpyAsync(F_target, h->w_Ft, KD * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    DevState s;
    TRY(read_state(h, &s));
    for (int j = 0; j < h->K; ++j) {
        if (log_ratio) log_ratio[j] = s.logr[j];
        if (log_u) log_u[j] = s.logu[j];
        if (delta_norm) delta_norm[j] = s.dnorm[j];
        if (accept) accept[j] = s.accept[j];
    }
    return LSD_OK;
}

int lsd_profile_window(lsd_handle *h, double *ms, int32_t n_phases) {
    if (!h || !ms || n_phases < 0) return LSD_EINVAL;
    DevState s;
    TRY(read_state(h, &s));
    const int Kp = h->stage_len ? h->stage_len : h->K;   // staged windows: the launch shape of one stage
    TRY(set_target_step(h, s.step + Kp));
    cudaEvent_t ev[LSD_N_PHASES + 1];
    for (int k = 0; k <= LSD_N_PHASES; ++k) CK(cudaEventCreate(&ev[k]));
    cudaStream_t st = h->stream;
    const int M = Kp * h->N;
    const PotDev &P = h->target.dev;
    // events in time order: t[0] Verlet lists t[1] draft t[2] neighbours ... t[8] commit t[9]; phase k < 8 is
    // t[k + 1] .. t[k + 2], the Verlet lists (phase 8) t[0] .. t[1]
    cudaEvent_t *t = ev;
    CK(cudaEventRecord(t[0], st));
    h->pipe_primed = false;
    lsd_handle::WinBufs &w0 = h->wb[0];
    if (!h->vplan.all_pairs) {   // as the handle's windows do: kept lists are rebuilt only when they must be
        if (h->list_reuse)
            enqueue_kept_lists(h, w0, st);
        else
            launch_verlet_build(h->vplan, h->q, h->species, h->geo, w0.vb, h->st, st);
    }
    CK(cudaEventRecord(t[1], st));
    launch_draft(h->grid_draft ? h->gplan : h->dplan, h->learned_small, Kp, h->geo, h->draft.dev, h->coef, h->vplan,
                 w0.vb, h->species, h->q, h->p, h->ec_dF, h->ec_on, h->st, w0.qmid, w0.pdraft, w0.Fd, w0.Fraw, w0.fix,
                 h->w_dEdX, st, nullptr, 0, h->dsync, 0, h->w_nbr, h->nbr_cap);
    CK(cudaEventRecord(t[2], st));
    if (h->vplan.all_pairs)
        launch_neigh_build(h->w_fix, M, h->geo, h->target.rmax2f, h->target.near2f, h->cap_near, h->cap_far,
                           h->near_keys, h->far_keys, h->n_near, h->n_far, h->st, st, &h->st->k_eff);
    else
        launch_neigh_list(h->w_fix, h->vbufs.vlist, h->vbufs.vcount, h->vplan.cap, M, h->geo, h->target.rmax2f,
                          h->target.near2f, h->cap_near, h->cap_far, h->near_keys, h->far_keys, h->n_near, h->n_far,
                          h->st, &h->st->k_eff, st);
    CK(cudaEventRecord(t[3], st));
    if (P.has_mlp) launch_desc(h->w_fix, h->near_keys, h->n_near, h->cap_near, M, h->geo, P, h->X, st, mom_for(h, h->target));
    CK(cudaEventRecord(t[4], st));
    if (P.has_mlp) enqueue_mlp(h, h->target, M, st);
    CK(cudaEventRecord(t[5], st));
    launch_pairgrad(h->w_fix, h->near_keys, h->n_near, h->far_keys, h->n_far, h->cap_near, h->cap_far, M, h->geo, P,
                    h->dEdX, h->pair_g, h->Fpart, h->E_lj, st, mom_for(h, h->target));
    CK(cudaEventRecord(t[6], st));
    launch_force_gather(h->near_keys, h->n_near, h->cap_near, M, h->N, P.has_mlp, h->pair_g, h->Fpart, h->E_lj,
                        h->E_mlp, h->w_Ft, nullptr, h->st, st);
    CK(cudaEventRecord(t[7], st));
    launch_transport_reduce(Kp, h->geo, h->coef, h->species, h->w_Fd, h->w_Ft, h->st, h->partials, &h->st->k_eff, st);
    CK(cudaEventRecord(t[8], st));
    launch_transport_commit(Kp, h->geo, h->coef, h->species, h->w_qmid, h->w_pdraft, h->w_Fd, h->w_Ft, h->w_Fraw,
                            h->ec_dF, h->ec_on, h->q, h->p, h->p_obabo, h->st, h->partials, &h->st->k_eff, st);
    CK(cudaEventRecord(t[9], st));
    CK(cudaGetLastError());
    TRY(wait_stream(h));
    for (int k = 0; k < LSD_N_PHASES && k < n_phases; ++k) {
        float e = 0.f;
        if (k < 8)
            CK(cudaEventElapsedTime(&e, t[k + 1], t[k + 2]));
        else
            CK(cudaEventElapsedTime(&e, t[0], t[1]));
        ms[k] = e;
    }
    for (int k = 0; k <= LSD_N_PHASES; ++k) cudaEventDestroy(ev[k]);
    TRY(read_state(h, &s));
    return check_err(s);
}

// The target's tensor-core MLP without any device allocation: the kernel's
// SiLU' scratch is a fixed array inside the library (see lsd_mlp_tc.cu), the
// caller passes the inputs and outputs.  For callers that own every device
// allocation themselves or cannot stall on cudaMalloc's implicit device
// synchronisation in a latency-critical loop.
int lsd_target_mlp_static_dev(lsd_handle *h, const float *X_dev, int32_t M, float *E_dev, float *dEdX_dev) {
    if (!h || !X_dev || !E_dev || !dEdX_dev || M < 1) return LSD_EINVAL;
    if (!h->target.tc_plan) return LSD_EUNSUPPORTED;
    return mlp_tc_static_launch(h->target.tc_plan, X_dev, M, h->target.dev, E_dev, dEdX_dev, h->target.tc_scales,
                                h->n_sm, &h->st->err, h->stream);
}

int lsd_query(const lsd_handle *h, int32_t *K, int32_t *n_atoms, int32_t *d_in, int32_t *nb_cap) {
    if (!h) return LSD_EINVAL;
    if (K) *K = h->K;
    if (n_atoms) *n_atoms = h->N;
    if (d_in) *d_in = h->target.dev.d0;
    if (nb_cap) *nb_cap = h->cap_near + h->cap_far;
    return LSD_OK;
}

// The launch sequences of enqueue_draft_buf, enqueue_verify_buf, enqueue_round
// and enqueue_plain, counted.
int lsd_launch_counts(const lsd_handle *h, int32_t *per_window, int32_t *per_round, int32_t *per_plain) {
    if (!h) return LSD_EINVAL;
    const bool lists = !h->vplan.all_pairs;
    const bool one_cell = h->vplan.nc[0] < 3 || h->vplan.nc[1] < 3 || h->vplan.nc[2] < 3;
    const int verlet = lists ? (one_cell ? 2 : 4) : 0;
    const int eval = 3 + (h->target.dev.has_mlp ? 2 : 0);   // neighbours, [descriptors, MLP,] pair gradients, gather
    const int nb = (h->N + transport_atoms_per_block(h->N) - 1) / transport_atoms_per_block(h->N);
    const int transport = nb == 1 ? 1 : 2;
    const int verify = eval + (h->train.capture_on ? 1 : 0) + transport;
    const int draft = verlet + 1;
    const int check = (lists && h->list_reuse) ? 1 : 0;   // the kept lists' verdict
    if (per_window) *per_window = check + draft + verify;
    // verify; spec_base; speculative draft; redraft (with its flag kernel in list mode)
    if (per_round) *per_round = verify + 1 + draft + (lists ? 1 : 0) + draft;
    if (per_plain) *per_plain = use_plain_fused(h) ? 0 : (lists ? 1 : 0) + verlet + 1 + eval + 1;
    return LSD_OK;
}

int lsd_stage_launch_counts(const lsd_handle *h, int32_t *first, int32_t *later) {
    if (!h) return LSD_EINVAL;
    int32_t w = 0;
    TRY(lsd_launch_counts(h, &w, nullptr, nullptr));
    const bool lists = !h->vplan.all_pairs;
    const bool one_cell = h->vplan.nc[0] < 3 || h->vplan.nc[1] < 3 || h->vplan.nc[2] < 3;
    const int verlet = lists ? (one_cell ? 2 : 4) : 0;
    if (first) *first = w;
    const int check = (lists && h->list_reuse) ? 1 : 0;
    if (later) *later = h->stage_len ? w - verlet - check : 0;   // a stage past the first rebuilds no lists
    return LSD_OK;
}

int lsd_set_list_reuse(lsd_handle *h, int32_t on) {
    if (!h) return LSD_EINVAL;
    if (on && h->pipe_on) return LSD_ESTATE;
    TRY(wait_stream(h));
    if (h->list_reuse != (on != 0)) destroy_graphs(h);
    h->list_reuse = on != 0;
    return LSD_OK;
}

int lsd_set_window_stages(lsd_handle *h, int32_t steps_per_stage) {
    if (!h || steps_per_stage < 0) return LSD_EINVAL;
    const int S = steps_per_stage < h->K ? steps_per_stage : 0;
    if (S && h->pipe_on) return LSD_ESTATE;
    TRY(wait_stream(h));
    if (S != h->stage_len) destroy_graphs(h);
    h->stage_len = S;
    // the draft's up-front noise buffer sized for its launches: S steps (or K); the cluster form only shrinks it
    const int steps = S ? S : h->K;
    h->gplan = h->gplan0;
    if (h->gplan0.ok) {
        DraftPlan g2 = h->gplan0;
        draft_plan_noise(g2, steps);
        if (g2.ok && draft_grid_fits(g2, h->learned_small, h->n_sm)) h->gplan = g2;
    }
    h->dplan = h->dplan0;
    DraftPlan d2 = h->dplan0;
    draft_plan_noise(d2, steps);
    if (d2.ok && d2.smem <= h->dplan0.smem) h->dplan = d2;
    return LSD_OK;
}

int lsd_set_angular_moments(lsd_handle *h, int32_t on) {
    if (!h) return LSD_EINVAL;
    if (on && !(h->target.dev.has_mlp && h->target.dev.n_ang)) return LSD_EUNSUPPORTED;
    TRY(wait_stream(h));
    if (on && !h->mom_on) {
        // the buffer was sized for one row when the handle chose the pair sums
        float *m = nullptr;
        TRY(dalloc(h, &m, (size_t)h->K * h->N * kMomRowFloats));
        h->mom = m;
    }
    if (h->mom_on != (on != 0)) destroy_graphs(h);   // the descriptor and pair-gradient launches are in the graphs
    h->mom_on = on != 0;
    return LSD_OK;
}

int lsd_get_angular_moments(const lsd_handle *h, int32_t *on) {
    if (!h || !on) return LSD_EINVAL;
    *on = (h->mom_on && h->target.dev.n_ang) ? 1 : 0;
    return LSD_OK;
}

int lsd_set_grid_draft(lsd_handle *h, int32_t on) {
    if (!h) return LSD_EINVAL;
    if (on && !h->gplan.ok) return LSD_EUNSUPPORTED;
    TRY(wait_stream(h));
    if (h->grid_draft != (on != 0)) destroy_graphs(h);   // the draft launch is part of the captured graphs
    h->grid_draft = on != 0;
    return LSD_OK;
}

int lsd_set_plain_fused(lsd_handle *h, int32_t on) {
    if (!h) return LSD_EINVAL;
    if (on && !h->pplan.ok) return LSD_EUNSUPPORTED;
    TRY(wait_stream(h));
    h->plain_fused = on != 0;
    return LSD_OK;
}

// ---- checkpoint / restore -------------------------------------------------
namespace {
constexpr uint64_t kCkptMagic = 0x4c53444350543032ull;   // "LSDCPT02"
struct CkptHeader {
    uint64_t magic;
    int64_t n_atoms, K, step, ec_on, n_weights, n_adam;
    uint64_t seed;
    int64_t integrator;   // LSD_ABOBA / LSD_OBABO
};
}  // namespace

int lsd_checkpoint(const lsd_handle *hc, void *buf, size_t *len) {
    if (!hc || !len) return LSD_EINVAL;
    lsd_handle *h = const_cast<lsd_handle *>(hc);
    const size_t D = 3 * (size_t)h->N;
    const size_t nw = h->draft.weights.size();
    const size_t nadam = train_adam_size(h->train);
    // q, p (the chain's own momentum: staggered under OBABO), EC cache, draft weights, Adam moments, OBABO output
    const size_t need = sizeof(CkptHeader) + 3 * D * sizeof(double) + D * sizeof(float) + nw * sizeof(float) +
                        2 * nadam * sizeof(float);
    if (!buf) {
        *len = need;
        return LSD_OK;
    }
    if (*len < need) {
        *len = need;
        return LSD_EINVAL;
    }
    CkptHeader hd{};
    hd.magic = kCkptMagic;
    hd.n_atoms = h->N;
    hd.K = h->K;
    hd.ec_on = h->ec_on;
    hd.n_weights = (int64_t)nw;
    hd.n_adam = (int64_t)nadam;
    hd.seed = h->seed;
    hd.integrator = h->coef.obabo ? LSD_OBABO : LSD_ABOBA;
    char *o = (char *)buf;
    DevState s;
    TRY(read_state(h, &s));
    hd.step = s.step;
    std::memcpy(o, &hd, sizeof(hd));
    double *qs = (double *)(o + sizeof(CkptHeader));
    CK(cudaMemcpyAsync(qs, h->q, D * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(qs + D, h->p, D * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    char *p = o + sizeof(CkptHeader) + 2 * D * sizeof(double);
    CK(cudaMemcpyAsync(p, h->ec_dF, D * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    p += D * sizeof(float);
    if (nw) std::memcpy(p, h->draft.weights.data(), nw * sizeof(float));
    p += nw * sizeof(float);
    TRY(train_adam_get(h->train, (float *)p, (float *)p + nadam));
    p += 2 * nadam * sizeof(float);
    CK(cudaMemcpyAsync(p, h->p_obabo, D * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    TRY(wait_stream(h));
    *len = need;
    return LSD_OK;
}

int lsd_restore(lsd_handle *h, const void *buf, size_t len) {
    if (!h || !buf || len < sizeof(CkptHeader)) return LSD_EINVAL;
    CkptHeader hd;
    std::memcpy(&hd, buf, sizeof(hd));
    const size_t D = 3 * (size_t)h->N;
    if (hd.magic != kCkptMagic || hd.n_atoms != h->N || hd.seed != h->seed ||
        hd.n_weights != (int64_t)h->draft.weights.size() || hd.n_adam != (int64_t)train_adam_size(h->train))
        return LSD_EINVAL;
    const size_t need = sizeof(CkptHeader) + 3 * D * sizeof(double) + D * sizeof(float) +
                        (size_t)hd.n_weights * sizeof(float) + 2 * (size_t)hd.n_adam * sizeof(float);
    if (len < need || (hd.integrator != LSD_ABOBA && hd.integrator != LSD_OBABO)) return LSD_EINVAL;
    const char *o = (const char *)buf + sizeof(CkptHeader);
    // the chain's own state, as saved (no re-entry into the OBABO frame)
    CK(cudaMemcpyAsync(h->q, o, D * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(h->p, (const double *)o + D, D * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    const long long stp = hd.step;
    CK(cudaMemcpyAsync(&h->st->step, &stp, sizeof(long long), cudaMemcpyHostToDevice, h->stream));
    h->pipe_primed = false;
    h->drafted = false;
    h->coef.obabo = hd.integrator == LSD_OBABO ? 1 : 0;
    {
        const char *po = o + 2 * D * sizeof(double) + D * sizeof(float) + (size_t)hd.n_weights * sizeof(float) +
                         2 * (size_t)hd.n_adam * sizeof(float);
        CK(cudaMemcpyAsync(h->p_obabo, po, D * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    }
    const char *p = o + 2 * D * sizeof(double);
    CK(cudaMemcpyAsync(h->ec_dF, p, D * sizeof(float), cudaMemcpyHostToDevice, h->stream));
    TRY(wait_stream(h));
    h->ec_on = (int)hd.ec_on;
    destroy_graphs(h);
    p += D * sizeof(float);
    if (hd.n_weights) {
        TRY(lsd_set_draft_weights(h, (const float *)p, (size_t)hd.n_weights));
    }
    p += (size_t)hd.n_weights * sizeof(float);
    TRY(train_adam_set(h->train, (const float *)p, (const float *)p + hd.n_adam));
    return LSD_OK;
}

// ---- frames and learned-draft training --------------------------------------
int lsd_set_frame_capture(lsd_handle *h, int64_t capacity) {
    if (!h || capacity < 0) return LSD_EINVAL;
    TRY(wait_stream(h));
    TRY(train_set_capture(h->train, capacity, h->N));
    destroy_graphs(h);
    return LSD_OK;
}

int lsd_frame_count(const lsd_handle *h, int64_t *n) {
    if (!h || !n) return LSD_EINVAL;
    return train_frame_count(const_cast<lsd_handle *>(h)->train, n, h->stream);
}

int lsd_set_online_training(lsd_handle *h, int64_t every_accepted, int32_t n_iters, float lr, int32_t frames_per_iter) {
    if (!h || every_accepted < 0 || n_iters < 0) return LSD_EINVAL;
    if (every_accepted > 0) {
        if (h->draft.p.kind != LSD_POT_LEARNED) return LSD_EINVAL;
        if (!h->train.capture_on) return LSD_ESTATE;   // frames are the training labels
    }
    DevState st;
    TRY(read_state(h, &st));
    h->online_every = every_accepted;
    h->online_iters = n_iters;
    h->online_lr = lr;
    h->online_fpi = frames_per_iter;
    h->online_base = st.committed - st.rejected;
    return LSD_OK;
}

int lsd_online_status(const lsd_handle *h, int64_t *retrains, float *last_loss) {
    if (!h) return LSD_EINVAL;
    if (retrains) *retrains = h->online_count;
    if (last_loss) *last_loss = h->online_loss;
    return LSD_OK;
}

int lsd_get_frames(lsd_handle *h, int64_t first, int64_t count, double *q, float *F) {
    if (!h || first < 0 || count < 0) return LSD_EINVAL;
    return train_get_frames(h->train, first, count, q, F, h->stream);
}

int lsd_train_draft(lsd_handle *h, int32_t n_iters, float lr, int32_t frames_per_iter, float *loss_out) {
    if (!h || n_iters < 0) return LSD_EINVAL;
    if (h->draft.p.kind != LSD_POT_LEARNED) return LSD_EINVAL;
    TRY(wait_stream(h));
    if (train_frame_fits(h->train)) {
        TRY(train_run(h->train, h->geo, h->draft.dev, h->species, n_iters, lr, frames_per_iter, loss_out, h->stream));
    } else {
        int64_t avail = 0;
        TRY(train_frame_count(h->train, &avail, h->stream));
        if (avail < 1) return LSD_ESTATE;
        const int fpi = (frames_per_iter <= 0 || frames_per_iter > avail) ? (int)avail : frames_per_iter;
        for (int it = 0; it < n_iters; ++it) {
            const long long frame0 = (h->train.iter * (long long)fpi) % avail;
            TRY(train_large_pass(h, h->train.fq, h->train.fF, frame0, avail, fpi, true, lr));
        }
        if (loss_out) {
            CK(cudaMemcpyAsync(loss_out, h->train.loss, sizeof(float), cudaMemcpyDeviceToHost, h->stream));
            CK(cudaStreamSynchronize(h->stream));
        }
    }
    // new weights -> draft MLP (FP32 master in the trainer)
    TRY(train_get_weights(h->train, h->draft.weights, h->stream));
    TRY(pot_upload(h, h->draft));
    destroy_graphs(h);
    return LSD_OK;
}

int lsd_force_match_dev(lsd_handle *h, const double *frames_q_dev, const float *frames_F_dev, int32_t n_frames,
                        float *loss_out, float *grad_dev) {
    if (!h || !frames_q_dev || !frames_F_dev || n_frames < 1) return LSD_EINVAL;
    if (h->draft.p.kind != LSD_POT_LEARNED) return LSD_EINVAL;
    TRY(wait_stream(h));
    if (train_frame_fits(h->train))
        return train_force_match(h->train, h->geo, h->draft.dev, h->species, frames_q_dev, frames_F_dev, n_frames,
                                 loss_out, grad_dev, h->stream);
    TRY(train_large_pass(h, frames_q_dev, frames_F_dev, 0, n_frames, n_frames, false, 0.f));
    if (grad_dev)
        CK(cudaMemcpyAsync(grad_dev, h->train.grad, h->train.n_weights * sizeof(float), cudaMemcpyDeviceToDevice,
                           h->stream));
    float l = 0.f;
    CK(cudaMemcpyAsync(&l, h->train.loss, sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    TRY(wait_stream(h));
    if (loss_out) *loss_out = l;
    DevState st;
    TRY(read_state(h, &st));
    return check_err(st);
}

}  // extern "C"
