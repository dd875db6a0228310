// lsd_mlp_tc.cu -- the per-atom energy MLP and its input gradient on the
// 5th-generation tensor cores (tcgen05, accumulators in tensor memory).  Same
// mathematics as lsd_mlp.cu:
//   forward  h_l = W_l a_{l-1} + b_l, a_l = SiLU(h_l), y = w_out.a_L + b_out
//   backward g_{L-1} = e'(y) w_out * SiLU'(h_{L-1}),
//            g_{l-1} = (g_l W_l) * SiLU'(h_{l-1}),  dE/dx = g_0 W_0
// Every layer is a GEMM D[128 x N] = A[128 x K] B[N x K]^T with the tile's 128
// rows in the 128 TMEM lanes:
//   forward  A = a_{l-1},  B = W_l   [W x din]  (N = W,    K = din)
//   backward A = g_l,      B = W_l^T [din x W]  (N = din,  K = W)
// Operand arithmetic, one template:
//   BF16     kind::f16, K = 16 per instruction;
//   TF32x3   FP32 targets: x = x_hi + x_lo (x_hi = tf32(x), x_lo = tf32(x - x_hi),
//            round to nearest); hi*hi + lo*hi + hi*lo in FP32 (the dropped
//            lo*lo is below 2^-22 of the product), K = 8.  B_hi and B_lo sit
//            one after the other in the stage, so one N = 2n instruction gives
//            A_hi B_hi (columns [0, n)) and A_hi B_lo ([n, 2n)), and a second,
//            N = n, adds A_lo B_hi to [0, n): two instructions per K step
//            instead of three; the epilogue adds the two column halves;
//   F16x3    FP32 targets, same split in FP16 (11 significant bits each) with
//            exact power-of-two scales (weights: max|W_l| near 2^14; every A
//            tensor: its calibrated |max| near 2^6, 1024x headroom below the
//            FP16 limit), K = 16: half the instructions of TF32x3 at the same
//            accuracy; the epilogue divides by the scales;
//   FP8      kind::f8f6f4, e4m3 with static per-tensor scales (weights: amax /
//            448 per layer; every activation and gradient tensor: a scale
//            calibrated once per handle), K = 32; the accumulator is rescaled
//            by s_A s_W in the epilogue.
// A lives in shared memory in the 128-byte-swizzled K-major layout, written by
// the epilogue of the previous GEMM.  B streams from global memory by TMA
// (2-D tiled copies, 128-byte swizzle), one 128-byte-wide K chunk per stage.
// Roles: warp 16 is the TMA producer and runs ahead through the whole GEMM
// sequence of the CTA's tiles, so the weights of the next GEMM land while the
// current epilogue runs; thread 0 issues the MMAs and commits them to
// mbarriers; warps 0..15 run the epilogues, warp w reading TMEM lane quarter
// w % 4 (rows 32 (w % 4) + lane) and the 32-column groups g = w / 4 + 4 k.
// SiLU'(h) stays in TMEM next to the accumulator when it fits, else in a
// per-CTA bf16 scratch that stays resident in L2.  The grid is persistent:
// one CTA per SM, looping over 128-row tiles.  Every mbarrier wait gives up
// after a bounded time and records an error.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "lsd.h"
#include "lsd_common.cuh"
#include "lsd_kernels.h"
#include "lsd_tc.cuh"

namespace lsd {

constexpr int kTcRows = 128;
constexpr int kPanelBytes = kTcRows * 128;           // one 128-byte-wide K panel of A: 16 KB
constexpr int kEpiWarps = 16;
constexpr int kEpiThreads = kEpiWarps * 32;
constexpr int kTcThreads = kEpiThreads + 32;         // + the TMA producer warp
constexpr uint32_t kTmemCols = 512;
constexpr int kStageBytes = 32 * 1024;               // one B stage: a 128-byte-wide K chunk of up to 256 rows
constexpr int kMiscBytes = 2048;                     // barriers, TMEM slot, head partial sums [3][128]
constexpr int kSmemBudget = 227 * 1024 - 1024;       // the opt-in maximum less the 1024-byte alignment slack

template <int OP> struct TcT;
// acc: TMEM columns reserved for the accumulator
template <> struct TcT<kTcBF16> {
    static constexpr int elem = 2, panel = 64, mmak = 16, copies = 1, maxk = 256, maxn = 256, acc = 256;
    static constexpr uint32_t fmt = tc::kFmtBF16;
};
template <> struct TcT<kTcTF32x3> {
    static constexpr int elem = 4, panel = 32, mmak = 8, copies = 2, maxk = 128, maxn = 128, acc = 256;
    static constexpr uint32_t fmt = tc::kFmtTF32;
};
template <> struct TcT<kTcF16x3> {
    static constexpr int elem = 2, panel = 64, mmak = 16, copies = 2, maxk = 128, maxn = 128, acc = 256;
    static constexpr uint32_t fmt = tc::kFmtF16;
};
template <> struct TcT<kTcFP8> {
    static constexpr int elem = 1, panel = 128, mmak = 32, copies = 1, maxk = 256, maxn = 256, acc = 256;
    static constexpr uint32_t fmt = tc::kFmtE4M3;
};
template <int OP> __host__ __device__ constexpr int tc_a_bytes() {
    return TcT<OP>::maxk / TcT<OP>::panel * kPanelBytes * TcT<OP>::copies;
}
template <int OP> __host__ __device__ constexpr int tc_stages() {
    return (kSmemBudget - tc_a_bytes<OP>() - kMiscBytes) / kStageBytes > 6
               ? 6
               : (kSmemBudget - tc_a_bytes<OP>() - kMiscBytes) / kStageBytes;
}
template <int OP> __host__ __device__ constexpr int tc_smem_bytes() {
    return 1024 + tc_a_bytes<OP>() + tc_stages<OP>() * kStageBytes + kMiscBytes;
}
static_assert(tc_smem_bytes<kTcBF16>() <= 227 * 1024, "BF16 shared memory");
static_assert(tc_smem_bytes<kTcTF32x3>() <= 227 * 1024, "TF32 shared memory");
static_assert(tc_smem_bytes<kTcFP8>() <= 227 * 1024, "FP8 shared memory");
static_assert(tc_smem_bytes<kTcF16x3>() <= 227 * 1024, "F16x3 shared memory");
static_assert(tc_stages<kTcTF32x3>() >= 2, "TF32 stages");

// Shared-memory addresses; per-stage ones are computed (a runtime-indexed
// array would live in local memory).
struct TcSm {
    uint32_t a;       // A panels; TF32 lo copy at a + tc_a_bytes / 2
    uint32_t b0;      // stage s at b0 + s kStageBytes; TF32: the lo chunk right after the N rows of the hi chunk
    uint32_t full0, empty0, done, tslot;
    float *ypart;     // [3][128] head partial sums of column blocks 1..3, then e'(y) per row
    __device__ __forceinline__ uint32_t b(int s) const { return b0 + (uint32_t)s * kStageBytes; }
    __device__ __forceinline__ uint32_t full(int s) const { return full0 + 8u * (uint32_t)s; }
    __device__ __forceinline__ uint32_t empty(int s) const { return empty0 + 8u * (uint32_t)s; }
};

struct TcMaps {
    CUtensorMap fwd[kMaxLayers][2];   // W_l   [W rows][din_p cols]; [1] = TF32 lo part
    CUtensorMap bwd[kMaxLayers][2];   // W_l^T [din_p rows][W cols]
};

// barrier 1: the epilogue warps only (the producer warp runs on its own)
__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kEpiThreads) : "memory"); }
__device__ __forceinline__ bool epi_and(bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.and.pred q, 1, %2, p;\n\tselp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(r)
        : "r"((uint32_t)v), "n"(kEpiThreads)
        : "memory");
    return r != 0;
}

// The MMAs of one GEMM, issued by one thread after the epilogue has published
// A.  chunk counts B chunks over the kernel (stage = chunk % S, use = chunk /
// S), in the producer's order.  Every chunk's stage is released to the
// producer by a commit; the last commit arrives on `done`.
template <int OP>
__device__ __forceinline__ bool tc_issue(const TcSm &S, int K, int N, uint32_t tmem, uint32_t chunk) {
    using T = TcT<OP>;
    constexpr int NS = tc_stages<OP>();
    const int nk = (K + T::panel - 1) / T::panel;
    tc::fence_after_sync();
    const uint32_t idesc = tc::idesc_f32acc(T::fmt, kTcRows, N);
    const uint32_t idesc2 = tc::idesc_f32acc(T::fmt, kTcRows, 2 * N);   // TF32: B_hi and B_lo stacked
    for (int kc = 0; kc < nk; ++kc) {
        const uint32_t c = chunk + kc;
        const int s = c % NS;
        if (!tc::mbar_wait(S.full(s), (c / NS) & 1)) return false;
        tc::fence_after_sync();
        const int kend = min(T::panel, K - kc * T::panel);
        // descriptors of the chunk's first K step; a K step advances the start address by mmak * elem bytes
        const uint64_t ad = tc::sdesc_sw128(S.a + kc * kPanelBytes), bd = tc::sdesc_sw128(S.b(s));
#pragma unroll
        for (int j = 0; j < T::panel / T::mmak; ++j) {
            if (j * T::mmak >= kend) break;
            const uint64_t step = (uint64_t)((j * T::mmak * T::elem) >> 4);
            const uint32_t acc = (kc | j) != 0;
            if (OP == kTcTF32x3) {
                const uint64_t alo = tc::sdesc_sw128(S.a + tc_a_bytes<OP>() / 2 + kc * kPanelBytes) + step;
                tc::mma_tf32(tmem, ad + step, bd + step, idesc2, acc);   // A_hi [B_hi; B_lo]
                tc::mma_tf32(tmem, alo, bd + step, idesc, 1u);            // + A_lo B_hi
            } else if (OP == kTcF16x3) {
                const uint64_t alo = tc::sdesc_sw128(S.a + tc_a_bytes<OP>() / 2 + kc * kPanelBytes) + step;
                tc::mma_f16(tmem, ad + step, bd + step, idesc2, acc);
                tc::mma_f16(tmem, alo, bd + step, idesc, 1u);
            } else if (OP == kTcFP8) {
                tc::mma_f8f6f4(tmem, ad + step, bd + step, idesc, acc);
            } else {
                tc::mma_f16(tmem, ad + step, bd + step, idesc, acc);
            }
        }
        tc::mma_commit(S.empty(s));
    }
    tc::mma_commit(S.done);
    return true;
}

// TF32 of x rounded to nearest, ties away from zero (the rounding of
// cvt.rna.tf32.f32) for finite x: half a TF32 ulp added to the magnitude bits,
// then the 13 bits below the TF32 mantissa cleared (a carry into the exponent
// is the correct rounding up).  Integer ALU work instead of a conversion.
__device__ __forceinline__ uint32_t tf32_rna(float x) { return (__float_as_uint(x) + 0x1000u) & 0xFFFFE000u; }
__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}
__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t *>(&h);
}
__device__ __forceinline__ uint32_t pack_f16(float a, float b) {
    const __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<const uint32_t *>(&h);
}
__device__ __forceinline__ uint32_t pack_e4m3(float a, float b, float c, float d) {
    const uint32_t lo = __nv_cvt_float2_to_fp8x2(make_float2(a, b), __NV_SATFINITE, __NV_E4M3);
    const uint32_t hi = __nv_cvt_float2_to_fp8x2(make_float2(c, d), __NV_SATFINITE, __NV_E4M3);
    return lo | (hi << 16);
}

// Writes 16 consecutive columns [c, c + 16) (c a multiple of 16) of row r of
// the A operand, in the operand format (FP8: v * qinv, saturating).
template <int OP>
__device__ __forceinline__ void store_a16(uint32_t a, int r, int c, const float (&v)[16], float qinv) {
    using T = TcT<OP>;
    const uint32_t pofs = (c / T::panel) * kPanelBytes;
    const int e0 = c % T::panel;   // element offset inside the 128-byte row
    if (OP == kTcBF16) {
#pragma unroll
        for (int q = 0; q < 2; ++q)
            st_shared_v4(a + pofs + tc::sw128_offset(r, e0 / 8 + q), pack_bf16(v[8 * q], v[8 * q + 1]),
                         pack_bf16(v[8 * q + 2], v[8 * q + 3]), pack_bf16(v[8 * q + 4], v[8 * q + 5]),
                         pack_bf16(v[8 * q + 6], v[8 * q + 7]));
    } else if (OP == kTcTF32x3) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            uint32_t h[4], l[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                h[e] = tf32_rna(v[4 * q + e]);
                l[e] = tf32_rna(v[4 * q + e] - __uint_as_float(h[e]));
            }
            const uint32_t off = pofs + tc::sw128_offset(r, e0 / 4 + q);
            st_shared_v4(a + off, h[0], h[1], h[2], h[3]);
            st_shared_v4(a + tc_a_bytes<OP>() / 2 + off, l[0], l[1], l[2], l[3]);
        }
    } else if (OP == kTcF16x3) {
        // scaled by qinv (a power of two); hi = x rounded to 11 significant bits
        // (exact in FP16 in its normal range), lo = FP16 of the exact remainder
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            uint32_t h[4], l[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float x0 = v[8 * q + 2 * e] * qinv, x1 = v[8 * q + 2 * e + 1] * qinv;
                const float h0 = __uint_as_float(tf32_rna(x0)), h1 = __uint_as_float(tf32_rna(x1));
                h[e] = pack_f16(h0, h1);
                l[e] = pack_f16(x0 - h0, x1 - h1);
            }
            const uint32_t off = pofs + tc::sw128_offset(r, e0 / 8 + q);
            st_shared_v4(a + off, h[0], h[1], h[2], h[3]);
            st_shared_v4(a + tc_a_bytes<OP>() / 2 + off, l[0], l[1], l[2], l[3]);
        }
    } else {
        st_shared_v4(a + pofs + tc::sw128_offset(r, e0 / 16),
                     pack_e4m3(v[0] * qinv, v[1] * qinv, v[2] * qinv, v[3] * qinv),
                     pack_e4m3(v[4] * qinv, v[5] * qinv, v[6] * qinv, v[7] * qinv),
                     pack_e4m3(v[8] * qinv, v[9] * qinv, v[10] * qinv, v[11] * qinv),
                     pack_e4m3(v[12] * qinv, v[13] * qinv, v[14] * qinv, v[15] * qinv));
    }
}

__device__ __forceinline__ float amax16(float m, const float (&v)[16]) {
#pragma unroll
    for (int i = 0; i < 16; ++i) m = fmaxf(m, fabsf(v[i]));
    return m;
}
// records a tensor's |max| (calibration): one atomic per warp
__device__ __forceinline__ void record_amax(float *amax, int slot, float m) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<int *>(amax) + slot, __float_as_int(m));
}

// The TMA producer: B chunks of every GEMM of the CTA's tiles, in the order
// the MMAs consume them, at most S stages ahead.  Before returning it waits
// for the landing of the copies it issued, so none is in flight at exit.
template <int OP>
__device__ void tc_producer(const TcSm &S, const TcMaps &maps, int M, const PotDev &P, int *err) {
    using T = TcT<OP>;
    constexpr int NS = tc_stages<OP>();
    const int W = P.width, L = P.n_layers, d0p = P.d0p;
    const int ntiles = (M + kTcRows - 1) / kTcRows;
    uint32_t c = 0;
    bool ok = true;
    auto gemm_chunks = [&](const CUtensorMap *m, int K, int N) {
        const int nk = (K + T::panel - 1) / T::panel;
        for (int kc = 0; kc < nk && ok; ++kc, ++c) {
            const int s = c % NS;
            if (c >= (uint32_t)NS && !tc::mbar_wait(S.empty(s), ((c / NS) - 1) & 1)) {
                ok = false;
                break;
            }
            tc::mbar_expect_tx(S.full(s), (uint32_t)T::copies * (uint32_t)N * 128u);
            tc::tma_load_2d(S.b(s), &m[0], kc * T::panel, 0, S.full(s));
            if (T::copies == 2) tc::tma_load_2d(S.b(s) + (uint32_t)N * 128u, &m[1], kc * T::panel, 0, S.full(s));
        }
    };
    for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        for (int l = 0; l < L && ok; ++l) gemm_chunks(maps.fwd[l], l == 0 ? d0p : W, W);
        for (int l = L - 1; l >= 0 && ok; --l) gemm_chunks(maps.bwd[l], W, l == 0 ? d0p : W);
    }
    const uint32_t first = c > (uint32_t)NS ? c - NS : 0u;
    for (uint32_t k = first; k < c; ++k)
        if (!tc::mbar_wait(S.full(k % NS), (k / NS) & 1)) ok = false;
    if (!ok) atomicOr(err, 8);
}

// scales (FP8): [l] A scale of forward GEMM l, [L + l] A scale of backward
// GEMM l, [2L + l] weight scale of layer l.  amax (calibration, may be null):
// |max| of the same A tensors, slots [l] and [L + l].
//
// The head's factor e'(y) is a per-row scalar and every backward step is
// linear in the gradient, so the backward chain runs on u_{L-1} = w_out *
// SiLU'(h_{L-1}) (written as the last forward epilogue's A, with no second
// pass over the tile) and e'(y) multiplies dE/dx in the last epilogue.
// SiLU'(h_l) is kept for l < L - 1 only.
template <int OP>
__global__ void __launch_bounds__(kTcThreads, 1)
    mlp_tc_kernel(const __grid_constant__ TcMaps maps, const float *__restrict__ X, int M, PotDev P,
                  float *__restrict__ E_mlp, float *__restrict__ dEdX, __nv_bfloat16 *__restrict__ scratch,
                  const float *__restrict__ scales, float *__restrict__ amax, int *__restrict__ err) {
    constexpr int ACC = TcT<OP>::acc;   // accumulator columns reserved in TMEM
    constexpr int NS = tc_stages<OP>();
    extern __shared__ uint8_t smraw[];
    const uint32_t base = (tc::smem_u32(smraw) + 1023u) & ~1023u;
    TcSm S;
    S.a = base;
    S.b0 = S.a + tc_a_bytes<OP>();
    S.full0 = S.b0 + NS * kStageBytes;
    S.empty0 = S.full0 + 8 * NS;
    S.done = S.empty0 + 8 * NS;
    S.tslot = S.done + 8;
    S.ypart = reinterpret_cast<float *>(smraw + (S.full0 + 512 - tc::smem_u32(smraw)));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int W = P.width, L = P.n_layers, d0p = P.d0p;
    if (tid == 0) {
        for (int st = 0; st < NS; ++st) {
            tc::mbar_init(S.full(st), 1);
            tc::mbar_init(S.empty(st), 1);
        }
        tc::mbar_init(S.done, 1);
        tc::mbar_fence_init();
    }
    if (warp == 0) {
        tc::tmem_alloc(S.tslot, kTmemCols);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    uint32_t tmem;
    asm volatile("ld.shared.b32 %0, [%1];" : "=r"(tmem) : "r"(S.tslot));
    if (warp == kEpiWarps) {
        if (lane == 0) tc_producer<OP>(S, maps, M, P, err);
    } else {
        const int quarter = warp & 3, cb = warp >> 2;
        const int r = 32 * quarter + lane;                               // row in the tile
        const uint32_t tacc = tmem + ((uint32_t)(32 * quarter) << 16);   // this warp's lanes, column 0
        const bool sp_tmem = ACC + (L - 1) * W <= (int)kTmemCols;        // SiLU' next to the accumulator
        __nv_bfloat16 *my_scr = scratch ? scratch + (size_t)blockIdx.x * (L - 1) * kTcRows * W : nullptr;
        auto sp_addr = [&](int l, int c) -> __nv_bfloat16 * { return my_scr + ((size_t)l * kTcRows + r) * W + c; };
        auto store_sp = [&](int l, int c, const float (&d)[16]) {
            if (sp_tmem) {
                tc::tmem_st16_async(tacc + ACC + l * W + c, d);   // completes by the wait at the epilogue's end
            } else {
                uint4 *o = reinterpret_cast<uint4 *>(sp_addr(l, c));
                o[0] = make_uint4(pack_bf16(d[0], d[1]), pack_bf16(d[2], d[3]), pack_bf16(d[4], d[5]),
                                  pack_bf16(d[6], d[7]));
                o[1] = make_uint4(pack_bf16(d[8], d[9]), pack_bf16(d[10], d[11]), pack_bf16(d[12], d[13]),
                                  pack_bf16(d[14], d[15]));
            }
        };
        // the accumulator's columns [c, c + 16) of an N-column GEMM (TF32: the sum of the two halves)
        auto load_acc = [&](int c, int N, float (&v)[16]) {
            if (OP == kTcTF32x3 || OP == kTcF16x3) {
                uint32_t a[16], b[16];   // both halves in flight, one wait
                tc::tmem_ld16_issue(tacc + c, a);
                tc::tmem_ld16_issue(tacc + N + c, b);
                tc::tmem_wait_ld();
#pragma unroll
                for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(a[i]) + __uint_as_float(b[i]);
            } else {
                tc::tmem_ld16(tacc + c, v);
            }
        };
        // SiLU' of 16 columns from the scratch: the raw bf16 words (fetched ahead of use), then unpacked
        auto fetch_sp = [&](int l, int c, uint4 (&u)[2]) {
            const uint4 *o = reinterpret_cast<const uint4 *>(sp_addr(l, c));
            u[0] = o[0];
            u[1] = o[1];
        };
        auto unpack_sp = [&](const uint4 (&u)[2], float (&d)[16]) {
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const uint32_t w4[4] = {u[q].x, u[q].y, u[q].z, u[q].w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const __nv_bfloat162 h2 = *reinterpret_cast<const __nv_bfloat162 *>(&w4[e]);
                    d[8 * q + 2 * e] = __low2float(h2);
                    d[8 * q + 2 * e + 1] = __high2float(h2);
                }
            }
        };
        // The epilogue's A stores become visible to the tensor core, then
        // thread 0 issues the next GEMM.  Lanes 1..31 of warp 0 wait at the
        // warp barrier meanwhile: spinning on an mbarrier in the same warp
        // would take issue turns from the issuing lane.
        uint32_t chunk = 0, gemm = 0;
        auto issue = [&](int K, int N) -> bool {
            tc::tmem_wait_st();   // this epilogue's SiLU' stores
            tc::fence_async_shared();
            tc::fence_before_sync();
            epi_sync();
            bool iok = true;
            if (warp == 0) {
                if (lane == 0) iok = tc_issue<OP>(S, K, N, tmem, chunk);
                __syncwarp();
            }
            chunk += (K + TcT<OP>::panel - 1) / TcT<OP>::panel;
            return iok;
        };
        auto wait_acc = [&](bool iok) -> bool {
            const bool w = tc::mbar_wait(S.done, gemm & 1);
            ++gemm;
            tc::fence_after_sync();
            return epi_and(iok && w);
        };
        // the descriptors come from the stream's previous kernel (the producer's
        // weight copies do not depend on it and start at once)
        pdl_wait();
        pdl_release();
        bool ok = true;
        constexpr bool kScaled = OP == kTcFP8 || OP == kTcF16x3;   // static per-tensor scales
        const float sc_x = kScaled ? scales[0] : 1.f;
        const int ntiles = (M + kTcRows - 1) / kTcRows;
        for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
            const int row = tile * kTcRows + r;
            const bool live = row < M;
            // input descriptors into the A panels
            float am = 0.f;
            for (int c = 16 * cb; c < d0p; c += 64) {
                float v[16];
                if (live) {
                    const float4 *src = reinterpret_cast<const float4 *>(X + (size_t)row * d0p + c);
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const float4 t = src[i];
                        v[4 * i] = t.x;
                        v[4 * i + 1] = t.y;
                        v[4 * i + 2] = t.z;
                        v[4 * i + 3] = t.w;
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < 16; ++i) v[i] = 0.f;
                }
                if (amax) am = amax16(am, v);
                store_a16<OP>(S.a, r, c, v, 1.f / sc_x);
            }
            if (amax) record_amax(amax, 0, am);
            // forward; the last layer's epilogue also writes the backward chain's first A
            float y = 0.f, dedy = 0.f;
            for (int l = 0; l < L; ++l) {
                const bool last = l == L - 1;
                ok = wait_acc(issue(l == 0 ? d0p : W, W));
                if (!ok) break;
                const float dq = kScaled ? scales[l] * scales[2 * L + l] : 1.f;
                const float qinv = kScaled ? 1.f / scales[last ? L + L - 1 : l + 1] : 1.f;
                const float *bl = layer_bias(P, l);
                am = 0.f;
                for (int c = 16 * cb; c < W; c += 64) {
                    float v[16], d[16];
                    load_acc(c, W, v);
                    const float4 *b4p = reinterpret_cast<const float4 *>(bl + c);
#pragma unroll
                    for (int i = 0; i < 16; i += 4) {
                        const float4 b4 = __ldg(b4p + i / 4);
                        silu_dsilu_fast(v[i] * dq + b4.x, v[i], d[i]);
                        silu_dsilu_fast(v[i + 1] * dq + b4.y, v[i + 1], d[i + 1]);
                        silu_dsilu_fast(v[i + 2] * dq + b4.z, v[i + 2], d[i + 2]);
                        silu_dsilu_fast(v[i + 3] * dq + b4.w, v[i + 3], d[i + 3]);
                    }
                    if (last) {
                        const float4 *w4p = reinterpret_cast<const float4 *>(P.wout + c);
#pragma unroll
                        for (int i = 0; i < 16; i += 4) {
                            const float4 w4 = __ldg(w4p + i / 4);
                            y += v[i] * w4.x + v[i + 1] * w4.y + v[i + 2] * w4.z + v[i + 3] * w4.w;
                            d[i] *= w4.x;
                            d[i + 1] *= w4.y;
                            d[i + 2] *= w4.z;
                            d[i + 3] *= w4.w;
                        }
                        if (amax) am = amax16(am, d);
                        store_a16<OP>(S.a, r, c, d, qinv);
                    } else {
                        store_sp(l, c, d);
                        if (amax) am = amax16(am, v);
                        store_a16<OP>(S.a, r, c, v, qinv);
                    }
                }
                if (amax) record_amax(amax, last ? L + L - 1 : l + 1, am);
                if (last && cb > 0) S.ypart[(cb - 1) * kTcRows + r] = y;
            }
            if (!ok) break;
            // backward; the head (energy, e'(y)) is finished while the first backward GEMM runs
            for (int l = L - 1; l >= 0; --l) {
                const int dout = l == 0 ? d0p : W;
                const bool iok = issue(W, dout);
                // the scratch's SiLU'(h_{l-1}) of this thread's first chunk, fetched while the GEMM runs; each
                // later chunk's is fetched while the previous one is processed (L2 latency off the chain)
                const bool sp_glob = l > 0 && !sp_tmem;
                uint4 spn[2] = {make_uint4(0u, 0u, 0u, 0u), make_uint4(0u, 0u, 0u, 0u)};
                if (sp_glob && 16 * cb < dout) fetch_sp(l - 1, 16 * cb, spn);
                if (l == L - 1) {
                    if (cb == 0) {
                        for (int b = 1; b < 4 && 16 * b < W; ++b) y += S.ypart[(b - 1) * kTcRows + r];
                        y += P.bout;
                        if (P.head == LSD_HEAD_LINEAR) {
                            if (live) E_mlp[row] = y;
                            dedy = 1.f;
                        } else {
                            const float t = tanhf(y);
                            if (live) E_mlp[row] = P.head_scale * t;
                            dedy = P.head_scale * (1.f - t * t);
                        }
                        S.ypart[r] = dedy;
                    }
                    epi_sync();
                    dedy = S.ypart[r];
                }
                ok = wait_acc(iok);
                if (!ok) break;
                const float dq = kScaled ? scales[L + l] * scales[2 * L + l] : 1.f;
                const float qinv = (kScaled && l > 0) ? 1.f / scales[L + l - 1] : 1.f;
                am = 0.f;
                for (int c = 16 * cb; c < dout; c += 64) {
                    float v[16];
                    uint4 spc[2] = {spn[0], spn[1]};
                    if (sp_glob && c + 64 < dout) fetch_sp(l - 1, c + 64, spn);
                    load_acc(c, dout, v);
                    if (l > 0) {
                        float d[16];
                        if (sp_tmem)
                            tc::tmem_ld16(tacc + ACC + (l - 1) * W + c, d);
                        else
                            unpack_sp(spc, d);
#pragma unroll
                        for (int i = 0; i < 16; ++i) v[i] *= dq * d[i];
                        if (amax) am = amax16(am, v);
                        store_a16<OP>(S.a, r, c, v, qinv);
                    } else if (live) {
                        const float f = dq * dedy;
                        float4 *dst = reinterpret_cast<float4 *>(dEdX + (size_t)row * d0p + c);
#pragma unroll
                        for (int i = 0; i < 4; ++i)
                            dst[i] = make_float4(v[4 * i] * f, v[4 * i + 1] * f, v[4 * i + 2] * f, v[4 * i + 3] * f);
                    }
                }
                if (amax && l > 0) record_amax(amax, L + l - 1, am);
            }
        }
        if (!ok && tid == 0) atomicOr(err, 8);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, kTmemCols);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct TcPlanImpl {
    int op;
    TcMaps maps;
};

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

// 2-D tensor [rows][cols] (cols contiguous) of the operand type; box = one
// 128-byte row of columns x box_rows rows, 128-byte swizzle.
static bool make_map(CUtensorMap *m, int op, const void *ptr, int rows, int cols, int box_rows) {
    auto fn = encode_fn();
    if (!fn) return false;
    const int elem = (op == kTcBF16 || op == kTcF16x3) ? 2 : (op == kTcTF32x3 ? 4 : 1);
    const CUtensorMapDataType dt = op == kTcBF16     ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                   : op == kTcF16x3  ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                   : op == kTcTF32x3 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                                     : CU_TENSOR_MAP_DATA_TYPE_UINT8;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)cols * elem};
    cuuint32_t box[2] = {(cuuint32_t)(128 / elem), (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    return fn(m, dt, 2, const_cast<void *>(ptr), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}

bool mlp_tc_supported(int op, const PotDev &P) {
    if (!P.has_mlp || P.width % 32 != 0 || P.n_layers > kMaxLayers || P.n_layers < 1 || !encode_fn()) return false;
    if (op == kTcTF32x3 || op == kTcF16x3)
        return P.width <= 128 && P.d0p <= 128 && 256 + (P.n_layers - 1) * P.width <= (int)kTmemCols;
    return P.width <= 256 && P.d0p <= 256;
}

void *mlp_tc_plan(int op, const PotDev &P, const TcWeights &w) {
    TcPlanImpl *pl = new TcPlanImpl();
    pl->op = op;
    bool ok = true;
    const int ncopy = (op == kTcTF32x3 || op == kTcF16x3) ? 2 : 1;
    for (int l = 0; l < P.n_layers && ok; ++l) {
        const int dinp = l == 0 ? P.d0p : P.width;
        for (int k = 0; k < ncopy && ok; ++k)
            ok = make_map(&pl->maps.fwd[l][k], op, w.wn[l][k], P.width, dinp, P.width) &&
                 make_map(&pl->maps.bwd[l][k], op, w.wt[l][k], dinp, P.width, dinp);
    }
    if (!ok) {
        delete pl;
        return nullptr;
    }
    return pl;
}

void mlp_tc_plan_free(void *plan) { delete (TcPlanImpl *)plan; }

int mlp_tc_plan_op(const void *plan) { return ((const TcPlanImpl *)plan)->op; }

size_t mlp_tc_smem_bytes(int op) {
    return op == kTcBF16     ? tc_smem_bytes<kTcBF16>()
           : op == kTcTF32x3 ? tc_smem_bytes<kTcTF32x3>()
           : op == kTcF16x3  ? tc_smem_bytes<kTcF16x3>()
                             : tc_smem_bytes<kTcFP8>();
}

// SiLU'(h_l) of the hidden layers but the last, per CTA, when it does not fit
// next to the accumulator in TMEM
size_t mlp_tc_scratch_elems(int op, const PotDev &P, int n_cta) {
    if (256 + (P.n_layers - 1) * P.width <= (int)kTmemCols) return 0;
    return (size_t)n_cta * (P.n_layers - 1) * kTcRows * P.width;
}

int mlp_tc_grid(int M, int n_sm) {
    const int ntiles = (M + kTcRows - 1) / kTcRows;
    return ntiles < n_sm ? ntiles : n_sm;
}

static void launch_grid(const TcPlanImpl *pl, int grid, const float *X, int M, const PotDev &P, float *E_mlp,
                        float *dEdX, __nv_bfloat16 *scratch, const float *scales, float *amax, int *err,
                        cudaStream_t s) {
    switch (pl->op) {
        case kTcBF16:
            launch_dependent(mlp_tc_kernel<kTcBF16>, grid, kTcThreads, tc_smem_bytes<kTcBF16>(), s, pl->maps, X, M, P,
                             E_mlp, dEdX, scratch, scales, amax, err);
            break;
        case kTcTF32x3:
            launch_dependent(mlp_tc_kernel<kTcTF32x3>, grid, kTcThreads, tc_smem_bytes<kTcTF32x3>(), s, pl->maps, X, M,
                             P, E_mlp, dEdX, scratch, scales, amax, err);
            break;
        case kTcF16x3:
            launch_dependent(mlp_tc_kernel<kTcF16x3>, grid, kTcThreads, tc_smem_bytes<kTcF16x3>(), s, pl->maps, X, M,
                             P, E_mlp, dEdX, scratch, scales, amax, err);
            break;
        default:
            launch_dependent(mlp_tc_kernel<kTcFP8>, grid, kTcThreads, tc_smem_bytes<kTcFP8>(), s, pl->maps, X, M, P,
                             E_mlp, dEdX, scratch, scales, amax, err);
            break;
    }
}

void launch_mlp_tc(const void *plan, const float *X, int M, const PotDev &P, float *E_mlp, float *dEdX,
                   __nv_bfloat16 *scratch, const float *scales, float *amax, int n_sm, int *err, cudaStream_t s) {
    launch_grid((const TcPlanImpl *)plan, mlp_tc_grid(M, n_sm), X, M, P, E_mlp, dEdX, scratch, scales, amax, err, s);
}

cudaError_t mlp_tc_setup() {
    cudaError_t e = cudaFuncSetAttribute(mlp_tc_kernel<kTcBF16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         tc_smem_bytes<kTcBF16>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(mlp_tc_kernel<kTcTF32x3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 tc_smem_bytes<kTcTF32x3>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(mlp_tc_kernel<kTcFP8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 tc_smem_bytes<kTcFP8>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(mlp_tc_kernel<kTcF16x3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 tc_smem_bytes<kTcF16x3>());
    return e;
}

// ---------------------------------------------------------------------------
// The same kernel for callers that cannot allocate device memory: its SiLU'
// scratch is this file-scope array (4 MiB, held by every device that loads the
// library until the process exits) instead of a slot the handle allocated.
// Nothing in it has to start at zero: each CTA writes a row's SiLU' values
// before reading them.  All calls share the array, so calls that overlap on
// the GPU (two streams, two handles) race on it.
// ---------------------------------------------------------------------------
constexpr size_t kStaticScratchBytes = (size_t)4 << 20;
constexpr size_t kStaticScratchElems = kStaticScratchBytes / sizeof(__nv_bfloat16);
static __device__ __align__(256) __nv_bfloat16 g_static_mlp_scratch[kStaticScratchElems];

constexpr int kStaticMaxDevices = 64;
static void *g_static_scratch_addr[kStaticMaxDevices];   // device address of the array, per device

size_t mlp_tc_static_scratch_bytes() { return kStaticScratchBytes; }

int mlp_tc_static_launch(const void *plan, const float *X, int M, const PotDev &P, float *E_mlp, float *dEdX,
                         const float *scales, int n_sm, int *err, cudaStream_t s) {
    const TcPlanImpl *pl = (const TcPlanImpl *)plan;
    const size_t per_cta = mlp_tc_scratch_elems(pl->op, P, 1);
    if (per_cta > kStaticScratchElems) return LSD_EINVAL;   // one tile's SiLU' does not fit the array
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kStaticMaxDevices) return LSD_ECUDA;
    if (!g_static_scratch_addr[dev]) {
        // set-up, once per device, with that device current: the host-side name
        // of the array is not a device address; ask the runtime for it
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_mlp_scratch) != cudaSuccess || !p) return LSD_ECUDA;
        g_static_scratch_addr[dev] = p;
    }
    int grid = mlp_tc_grid(M, n_sm);
    if (per_cta > 0) {
        const int cap = (int)(kStaticScratchElems / per_cta);
        if (grid > cap) grid = cap;
    }
    launch_grid(pl, grid, X, M, P, E_mlp, dEdX, per_cta > 0 ? (__nv_bfloat16 *)g_static_scratch_addr[dev] : nullptr,
                scales, nullptr, err, s);
    return cudaGetLastError() == cudaSuccess ? LSD_OK : LSD_ECUDA;
}

}  // namespace lsd
