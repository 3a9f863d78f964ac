// mlp_internal.h — state of the learned initial-state proposal (host side).
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

#include "../../include/firert.h"
#include "internal.cuh"

struct fire_mlp {
  fire_ctx_t *ctx;
  firert::KTables ctx_t;
  firert::KConfig ctx_c;
  int K, H, Din, n_out;
  int have_stats;
  int64_t step, sample_next;
  long long cap;
  // FP32 master weights and biases, Adam moments
  float *W1, *W2, *W3, *b1, *b2, *b3;
  float *mW1, *vW1, *mW2, *vW2, *mW3, *vW3, *mb1, *vb1, *mb2, *vb2, *mb3, *vb3;
  // bf16 copies for the tensor cores and their transposes
  __nv_bfloat16 *W1b, *W2b, *W3b, *W1T, *W2T, *W3T;
  // input standardisation
  float *mean, *istd;
  // per-batch activations and gradients
  __nv_bfloat16 *x, *xT, *h1, *h1T, *h2, *h2T, *dy, *dyT, *dh2, *dh2T, *dh1, *dh1T;
  float *z, *tgt, *msk, *rad;
  float *gW1, *gW2, *gW3T, *gb1, *gb2, *gb3, *loss;
  int *err;
};

// tables and default solver constants of a context (api.cu)
void fire_ctx_tables(const fire_ctx_t *ctx, firert::KTables *t, firert::KConfig *c);
