// Conv-net preconditioner object shared by convnet.cu and learned.cu.
#pragma once

#include "plan.cuh"
#include "solve.cuh"

#define HQS_NET_HIDDEN 32

struct hqs_net_s {
    float* params = nullptr;   // [W1 b1 W2 b2 W3 b3 W4 b4], W[o][i][3][3]
    float* grads = nullptr;
    float* m = nullptr;        // Adam moments
    float* v = nullptr;
    int adam_t = 0;
    // HQS_PREC_BF16X3: the 32 -> 32 layers' forward and input-gradient convolutions
    // on the tensor cores; HQS_PREC_FP32: every convolution on the FP32 cores
    int precision = HQS_PREC_BF16X3;
    unsigned* dev_err = nullptr;   // HQS_DEVERR_* bits of the tensor-core convolutions
    // activations and gradient scratch, grown on demand
    float* act[4] = {nullptr, nullptr, nullptr, nullptr};
    float* dbuf[2] = {nullptr, nullptr};
    float* part = nullptr;     // per-tile weight-gradient partials
    double* loss_n = nullptr;
    size_t cap_pix = 0, cap_tiles = 0;
    int cap_n = 0;
    // inference buffers of the preconditioner (n x n)
    float2* zdc = nullptr;
    float* planar = nullptr;
    double* scal = nullptr;
    int cap_img = 0;
};

int net_num_params();
int net_forward(hqs_net_s* net, const float* x, float* out, int N, int H, int Wd, cudaStream_t st);
int net_check(hqs_net_s* net, cudaStream_t st);
