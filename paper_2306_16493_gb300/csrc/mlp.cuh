// Learned q-proposal network (internal): a 9 -> 128 -> 128 -> 128 -> 1 perceptron with SiLU
// hidden activations, BF16 weights and FP32 arithmetic.  The paper has no learned part; the
// network only shapes the proposal of an importance-sampled estimate of the q sum of the
// SERTA rate (Sec. II C, Eq. 10), which stays unbiased whatever the network outputs.
#pragma once

#include "epwi_internal.cuh"

#include <vector>

namespace mlp {
constexpr int kIn = 9;
constexpr int kHid = 128;
// parameter blocks, in storage order
constexpr int64_t oW1 = 0;                          // [128][9]
constexpr int64_t ob1 = oW1 + kHid * kIn;           // [128]
constexpr int64_t oW2 = ob1 + kHid;                 // [128][128]
constexpr int64_t ob2 = oW2 + kHid * kHid;
constexpr int64_t oW3 = ob2 + kHid;                 // [128][128]
constexpr int64_t ob3 = oW3 + kHid * kHid;
constexpr int64_t ow4 = ob3 + kHid;                 // [128]
constexpr int64_t ob4 = ow4 + kHid;                 // [1]
constexpr int64_t kNParam = ob4 + 1;
constexpr double kEScale = 0.25;                    // eV, scale of the energy input
constexpr int kMaxBatch = 1 << 16;                  // rows of one training step
}  // namespace mlp

// Step-dependent scalars of one training step (graph-replayed training).
struct StepParams {
    int64_t i0;                       // first position of the batch in the epoch's permutation
    uint64_t a, b;                    // permutation i -> (a i + b) mod n
    float lr, bc1, bc2;               // Adam step size and bias corrections 1 - beta^t
    float pad;
};

// Network state kept in the context.
struct MlpState {
    bool ready = false;
    int64_t step = 0;                 // Adam steps taken
    double out_scale = 1.0, out_shift = 0.0;   // log t = scale * yhat + shift
    DevBuf master;                    // float [NP] FP32 master weights
    DevBuf w;                         // float [NP] BF16-rounded weights (the forward's values)
    DevBuf wbf;                       // uint16 [NP] the same as bf16 bit patterns
    DevBuf m, v, grad;                // float [NP] Adam moments, gradient
    DevBuf part;                      // float split-batch weight-gradient partials
    DevBuf act;                       // float activations of one batch
    DevBuf lossbuf;                   // double [..] per-block squared residual sums
    // training set
    int64_t n_train = 0;
    DevBuf X, Y;                      // float [n][9], float [n] normalised log targets
    DevBuf T64;                       // double [n] raw targets
    DevBuf ids;                       // int4 [n] {ik, iq, band, mode}
    DevBuf bx, by;                    // batch gather
    DevBuf err;                       // int: timed-out waits of the tensor-core inference
    void release() {
        DevBuf *all[] = {&master, &w, &wbf, &m, &v, &grad, &part, &act, &lossbuf,
                         &X, &Y, &T64, &ids, &bx, &by, &err};
        for (DevBuf *b : all) b->release();
        ready = false;
    }
};

// Kernels of mlp.cu (host launchers).
void mlp_init(epwi_ctx *c, uint64_t seed);
void mlp_set_master(epwi_ctx *c, const float *host_params);
void mlp_forward(epwi_ctx *c, int64_t n, const float *X, float *yhat);
double mlp_loss_grad(epwi_ctx *c, int64_t n, const float *X, const float *Y,
                     bool want_loss = true);
double mlp_dataset_loss(epwi_ctx *c);
void mlp_train_graph(epwi_ctx *c, const std::vector<StepParams> &steps, int64_t B);
// mlp_tc.cu: the same forward pass on the tensor cores (BF16 activations between layers)
int mlp_forward_tc(epwi_ctx *c, int64_t n, const float *X, float *y, int *err_dev);
// tensor-core forward with its error check (throws EPWI_ETIMEOUT)
void mlp_forward_fast(epwi_ctx *c, int64_t n, const float *X, float *y);

// learned.cu
void mlp_train(epwi_ctx *c, double T, double mu, double eta, double emin, double emax,
               const epwi_mlp_train_options &o, double *final_loss);
void run_is(epwi_ctx *c, double T, double mu, double eta, double emin, double emax,
            int64_t S, double alpha, int stride, int proposal, uint64_t seed);
