// lsd_train.h -- learned-draft frames and force-matching training (internal).
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "lsd_common.cuh"

namespace lsd {

struct TrainState {
    bool enabled = false;        // the draft is a learned MLP
    int N = 0, d0 = 0, W = 0, S = 0, n_rbf = 0;
    size_t n_weights = 0;
    // frame ring buffer (positions FP64, target forces FP32)
    bool capture_on = false;
    long long capacity = 0;
    long long start_verified = 0; // verified-steps counter when capture started
    int K = 0;
    double *fq = nullptr;
    float *fF = nullptr;
    // FP32 master weights (packed like the ABI) and Adam moments
    float *w = nullptr, *m = nullptr, *v = nullptr;
    float *grad_frames = nullptr;   // [max_frames][n_weights]
    float *loss_frames = nullptr;   // [max_frames]
    float *grad = nullptr;          // [n_weights]
    float *loss = nullptr;          // [1]
    int max_frames = 0;
    // frames larger than one block: per-row workspace of one frame
    float *lH = nullptr, *lT = nullptr, *lV = nullptr, *lFd = nullptr, *lloss = nullptr, *lpart = nullptr;
    float4 *lres = nullptr;
    long long adam_t = 0;
    long long iter = 0;
    DevState *st = nullptr;
};

int train_init(TrainState &t, const PotDev &P, const std::vector<float> &weights, int N);
void train_free(TrainState &t);
int train_set_weights(TrainState &t, const std::vector<float> &w);
int train_get_weights(TrainState &t, std::vector<float> &w, cudaStream_t s);
int train_set_capture(TrainState &t, long long capacity, int N);
int train_frame_count(TrainState &t, int64_t *n, cudaStream_t s);
int train_get_frames(TrainState &t, long long first, long long count, double *q, float *F, cudaStream_t s);
void enqueue_frame_capture(TrainState &t, const double *w_qmid, const float *w_Ft, int K, int N, DevState *st,
                           const int *keff, cudaStream_t s, int j0 = 0);   // window steps j0 .. K - 1
size_t train_adam_size(const TrainState &t);
int train_adam_get(TrainState &t, float *m, float *v);
int train_adam_set(TrainState &t, const float *m, const float *v);
int train_run(TrainState &t, const Geo &g, const PotDev &P, const int *species, int n_iters, float lr,
              int frames_per_iter, float *loss_out, cudaStream_t s);
// frames larger than one block (the caller runs lists, descriptors, pair gradients and the gather)
bool train_frame_fits(const TrainState &t);
int train_large_bufs(TrainState &t, int n_frames);
void launch_fm_mlp(const TrainState &t, const float *X, int d0p, float *G, cudaStream_t s);
void launch_fm_frame_grad(const TrainState &t, const uint4 *fix, const int *near_keys, const int *n_near, int cap,
                          const Geo &g, const PotDev &P, const float *X, int d0p, const float *Fstar, float scale,
                          int frame_index, cudaStream_t s);
void launch_fm_reduce_adam(TrainState &t, int n_frames, bool adam, float lr, cudaStream_t s);
int train_force_match(TrainState &t, const Geo &g, const PotDev &P, const int *species, const double *fq,
                      const float *fF, int n_frames, float *loss_out, float *grad_dev, cudaStream_t s);

}  // namespace lsd
