// mlp.cu — host orchestration of the learned initial-state proposal: weights,
// Adam state, training steps (synthesiser -> three forward GEMMs -> loss
// gradient -> weight/input-gradient GEMMs -> Adam), inference in chunks, and
// a checksummed checkpoint. Every product runs on the tensor cores
// (kernels_gemm.cu); every element-wise step is a kernel (kernels_mlp.cu).
#include <stdio.h>
#include <string.h>

#include <new>

#include "../../include/firert.h"
#include "internal.cuh"
#include "mlp_internal.h"

using namespace firert;

namespace firert {
cudaError_t launch_mlp_input(const float *rad, long long n, int nb, int Din, const float *mean,
                             const float *istd, __nv_bfloat16 *x, __nv_bfloat16 *xT, long long ldT,
                             cudaStream_t st);
cudaError_t launch_mlp_synth(const KTables &t, const KConfig &c, long long B, long long sample0,
                             unsigned long long seed, float pfire, float nrel, float nabs,
                             const float *mean, const float *istd, int Din, __nv_bfloat16 *x,
                             __nv_bfloat16 *xT, float *tgt, float *msk, float *rad_out,
                             cudaStream_t st);
cudaError_t launch_mlp_lossgrad(const float *z, const float *tgt, const float *msk, long long B,
                                int n_out, __nv_bfloat16 *dy, __nv_bfloat16 *dyT, float *loss,
                                cudaStream_t st);
cudaError_t launch_rowsum(const __nv_bfloat16 *in, int rows, long long cols, float *out, cudaStream_t st);
cudaError_t launch_adam(float *W, const float *G, int gT, float *m, float *v, int R, int Cc, float lr,
                        int step, __nv_bfloat16 *Wb, __nv_bfloat16 *WbT, cudaStream_t st);
cudaError_t launch_mlp_to_init(const float *z, long long n, int K, const KConfig &c, float *init,
                               cudaStream_t st);
cudaError_t launch_colstats(const float *rad, long long B, int nb, float *mean, float *istd,
                            cudaStream_t st);
cudaError_t launch_init_weights(float *W, long long n, float s, unsigned long long seed,
                                unsigned long long sid, cudaStream_t st);
cudaError_t launch_to_bf16(const float *W, int R, int Cc, __nv_bfloat16 *Wb, __nv_bfloat16 *WbT,
                           cudaStream_t st);
}  // namespace firert

namespace {

#define MCK(call)                                               \
  do {                                                          \
    cudaError_t e_ = (call);                                    \
    if (e_ != cudaSuccess)                                      \
      return e_ == cudaErrorMemoryAllocation ? FIRE_ERR_NOMEM : FIRE_ERR_CUDA; \
  } while (0)

template <class T>
cudaError_t dalloc(T **p, size_t n) {
  return dev_malloc((void **)p, n * sizeof(T));
}

GemmArgs gemm(const __nv_bfloat16 *A, long long lda, const __nv_bfloat16 *B, long long ldb, int M,
              int N, int K, int epi) {
  GemmArgs g;
  memset(&g, 0, sizeof(g));
  g.A = A;
  g.B = B;
  g.lda = lda;
  g.ldb = ldb;
  g.M = M;
  g.N = N;
  g.K = K;
  g.epi = epi;
  return g;
}

uint64_t fnv1a(const void *p, size_t n, uint64_t h) {
  const unsigned char *b = (const unsigned char *)p;
  for (size_t i = 0; i < n; i++) {
    h ^= b[i];
    h *= 1099511628211ull;
  }
  return h;
}

}  // namespace

void fire_mlp_free_buffers(fire_mlp *m) {
  void *ptrs[] = {m->W1, m->W2, m->W3, m->b1, m->b2, m->b3, m->mW1, m->vW1, m->mW2, m->vW2,
                  m->mW3, m->vW3, m->mb1, m->vb1, m->mb2, m->vb2, m->mb3, m->vb3, m->W1b, m->W2b,
                  m->W3b, m->W1T, m->W2T, m->W3T, m->mean, m->istd, m->x, m->xT, m->h1, m->h1T,
                  m->h2, m->h2T, m->z, m->tgt, m->msk, m->dy, m->dyT, m->dh2, m->dh2T, m->dh1,
                  m->dh1T, m->gW1, m->gW2, m->gW3T, m->gb1, m->gb2, m->gb3, m->loss, m->err,
                  m->rad};
  for (void *p : ptrs) dev_free(p);
}

fire_status_t fire_mlp_reserve(fire_mlp *m, long long B) {
  if (B <= m->cap) return FIRE_OK;
  void *old[] = {m->x, m->xT, m->h1, m->h1T, m->h2, m->h2T, m->z, m->tgt, m->msk, m->dy, m->dyT,
                 m->dh2, m->dh2T, m->dh1, m->dh1T, m->rad};
  for (void *p : old) dev_free(p);
  const int Din = m->Din, H = m->H;
  m->cap = 0;
  MCK(dalloc(&m->x, (size_t)B * Din));
  MCK(dalloc(&m->xT, (size_t)B * Din));
  MCK(dalloc(&m->h1, (size_t)B * H));
  MCK(dalloc(&m->h1T, (size_t)B * H));
  MCK(dalloc(&m->h2, (size_t)B * H));
  MCK(dalloc(&m->h2T, (size_t)B * H));
  MCK(dalloc(&m->z, (size_t)B * 16));
  MCK(dalloc(&m->tgt, (size_t)B * 16));
  MCK(dalloc(&m->msk, (size_t)B * 16));
  MCK(dalloc(&m->dy, (size_t)B * 16));
  MCK(dalloc(&m->dyT, (size_t)B * 16));
  MCK(dalloc(&m->dh2, (size_t)B * H));
  MCK(dalloc(&m->dh2T, (size_t)B * H));
  MCK(dalloc(&m->dh1, (size_t)B * H));
  MCK(dalloc(&m->dh1T, (size_t)B * H));
  MCK(dalloc(&m->rad, (size_t)B * m->ctx_t.nb));
  m->cap = B;
  return FIRE_OK;
}

// refresh the bf16 copies (and transposes) of the master weights
static fire_status_t refresh_bf16(fire_mlp *m, cudaStream_t st) {
  MCK(launch_to_bf16(m->W1, m->H, m->Din, m->W1b, m->W1T, st));
  MCK(launch_to_bf16(m->W2, m->H, m->H, m->W2b, m->W2T, st));
  MCK(launch_to_bf16(m->W3, 16, m->H, m->W3b, m->W3T, st));
  return FIRE_OK;
}

// forward through the three layers for B rows of m->x (bf16 inputs)
static fire_status_t forward_rows(fire_mlp *m, long long B, bool keep_T, cudaStream_t st) {
  const int Din = m->Din, H = m->H;
  GemmArgs g1 = gemm(m->x, Din, m->W1b, Din, (int)B, H, Din, EPI_BIAS_RELU);
  g1.bias = m->b1;
  g1.Cb = m->h1;
  g1.ldcb = H;
  if (keep_T) { g1.CbT = m->h1T; g1.ldcbT = B; }
  g1.err = m->err;
  MCK(launch_gemm(g1, st));
  GemmArgs g2 = gemm(m->h1, H, m->W2b, H, (int)B, H, H, EPI_BIAS_RELU);
  g2.bias = m->b2;
  g2.Cb = m->h2;
  g2.ldcb = H;
  if (keep_T) { g2.CbT = m->h2T; g2.ldcbT = B; }
  g2.err = m->err;
  MCK(launch_gemm(g2, st));
  GemmArgs g3 = gemm(m->h2, H, m->W3b, H, (int)B, 16, H, EPI_BIAS_TANH);
  g3.bias = m->b3;
  g3.Cf = m->z;
  g3.ldc = 16;
  g3.err = m->err;
  MCK(launch_gemm(g3, st));
  return FIRE_OK;
}

// backward of the masked MSE for the rows in m->x / m->tgt / m->msk:
// gradients into gW1 [H][Din], gb1, gW2 [H][H], gb2, gW3T [H][16], gb3
static fire_status_t backward_rows(fire_mlp *m, long long B, cudaStream_t st) {
  const int Din = m->Din, H = m->H;
  MCK(cudaMemsetAsync(m->loss, 0, sizeof(float), st));
  MCK(launch_mlp_lossgrad(m->z, m->tgt, m->msk, B, m->n_out, m->dy, m->dyT, m->loss, st));
  // dW3^T [H][16] = h2^T dy ; K = B
  GemmArgs a = gemm(m->h2T, B, m->dyT, B, H, 16, (int)B, EPI_F32);
  a.Cf = m->gW3T;
  a.ldc = 16;
  a.err = m->err;
  MCK(launch_gemm(a, st));
  // dh2 = (dy W3) * (h2 > 0) ; B = W3^T [H][16]
  GemmArgs b = gemm(m->dy, 16, m->W3T, 16, (int)B, H, 16, EPI_RELU_MASK);
  b.mask = m->h2;
  b.ldm = H;
  b.Cb = m->dh2;
  b.ldcb = H;
  b.CbT = m->dh2T;
  b.ldcbT = B;
  b.err = m->err;
  MCK(launch_gemm(b, st));
  // dW2 [H][H] = dh2^T h1
  GemmArgs c = gemm(m->dh2T, B, m->h1T, B, H, H, (int)B, EPI_F32);
  c.Cf = m->gW2;
  c.ldc = H;
  c.err = m->err;
  MCK(launch_gemm(c, st));
  // dh1 = (dh2 W2) * (h1 > 0) ; B = W2^T [H(in)][H(out)]
  GemmArgs d = gemm(m->dh2, H, m->W2T, H, (int)B, H, H, EPI_RELU_MASK);
  d.mask = m->h1;
  d.ldm = H;
  d.Cb = m->dh1;
  d.ldcb = H;
  d.CbT = m->dh1T;
  d.ldcbT = B;
  d.err = m->err;
  MCK(launch_gemm(d, st));
  // dW1 [H][Din] = dh1^T x
  GemmArgs e = gemm(m->dh1T, B, m->xT, B, H, Din, (int)B, EPI_F32);
  e.Cf = m->gW1;
  e.ldc = Din;
  e.err = m->err;
  MCK(launch_gemm(e, st));
  MCK(launch_rowsum(m->dyT, 16, B, m->gb3, st));
  MCK(launch_rowsum(m->dh2T, H, B, m->gb2, st));
  MCK(launch_rowsum(m->dh1T, H, B, m->gb1, st));
  return FIRE_OK;
}

extern "C" {

fire_status_t fire_mlp_create(fire_mlp_t **out, fire_ctx_t *ctx, int32_t hidden, uint64_t seed) {
  if (!out || !ctx) return FIRE_ERR_ARG;
  *out = nullptr;
  if (hidden < 16 || hidden > 1024 || (hidden & 15)) return FIRE_ERR_SHAPE;
  fire_mlp *m = new (std::nothrow) fire_mlp();
  if (!m) return FIRE_ERR_NOMEM;
  memset(m, 0, sizeof(*m));
  fire_ctx_tables(ctx, &m->ctx_t, &m->ctx_c);
  m->ctx = ctx;
  m->K = m->ctx_t.K;
  m->H = hidden;
  m->Din = (m->ctx_t.nb + 15) & ~15;
  m->n_out = m->K + 6;
  const int Din = m->Din, H = m->H;
  fire_status_t st = FIRE_OK;
#define MA(p, n) if (st == FIRE_OK && dalloc(&m->p, (size_t)(n)) != cudaSuccess) st = FIRE_ERR_NOMEM
  MA(W1, H * Din); MA(W2, H * H); MA(W3, 16 * H); MA(b1, H); MA(b2, H); MA(b3, 16);
  MA(mW1, H * Din); MA(vW1, H * Din); MA(mW2, H * H); MA(vW2, H * H); MA(mW3, 16 * H); MA(vW3, 16 * H);
  MA(mb1, H); MA(vb1, H); MA(mb2, H); MA(vb2, H); MA(mb3, 16); MA(vb3, 16);
  MA(W1b, H * Din); MA(W2b, H * H); MA(W3b, 16 * H); MA(W1T, H * Din); MA(W2T, H * H); MA(W3T, 16 * H);
  MA(mean, Din); MA(istd, Din); MA(gW1, H * Din); MA(gW2, H * H); MA(gW3T, 16 * H);
  MA(gb1, H); MA(gb2, H); MA(gb3, 16); MA(loss, 1); MA(err, 1);
#undef MA
  if (st != FIRE_OK) {
    fire_mlp_free_buffers(m);
    delete m;
    return st;
  }
  cudaStream_t s = 0;
  // He-uniform initialisation from the counter stream; zero biases and moments
  launch_init_weights(m->W1, (long long)H * Din, sqrtf(6.f / Din), seed, 11, s);
  launch_init_weights(m->W2, (long long)H * H, sqrtf(6.f / H), seed, 12, s);
  launch_init_weights(m->W3, 16LL * H, sqrtf(6.f / H), seed, 13, s);
  void *zero[] = {m->b1, m->b2, m->b3, m->mW1, m->vW1, m->mW2, m->vW2, m->mW3, m->vW3,
                  m->mb1, m->vb1, m->mb2, m->vb2, m->mb3, m->vb3, m->err};
  size_t zn[] = {(size_t)H, (size_t)H, 16, (size_t)H * Din, (size_t)H * Din, (size_t)H * H,
                 (size_t)H * H, 16u * H, 16u * H, (size_t)H, (size_t)H, (size_t)H, (size_t)H, 16, 16, 1};
  for (int i = 0; i < 16; i++) cudaMemsetAsync(zero[i], 0, zn[i] * 4, s);
  // input standardisation: identity until statistics are gathered
  {
    float *h = new float[2 * Din];
    for (int i = 0; i < Din; i++) { h[i] = 0.f; h[Din + i] = 1.f; }
    cudaMemcpy(m->mean, h, Din * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(m->istd, h + Din, Din * 4, cudaMemcpyHostToDevice);
    delete[] h;
  }
  st = refresh_bf16(m, s);
  if (st == FIRE_OK && cudaDeviceSynchronize() != cudaSuccess) st = FIRE_ERR_CUDA;
  if (st != FIRE_OK) {
    fire_mlp_free_buffers(m);
    delete m;
    return st;
  }
  *out = m;
  return FIRE_OK;
}

void fire_mlp_destroy(fire_mlp_t *m) {
  if (!m) return;
  fire_mlp_free_buffers(m);
  delete m;
}

fire_status_t fire_mlp_train(fire_mlp_t *m, const fire_mlp_train_cfg_t *cfg, float *loss_host,
                             fire_stream_t stream) {
  if (!m || !cfg || cfg->steps < 0 || cfg->batch < 128 || (cfg->batch & 127) || !(cfg->lr >= 0.f))
    return FIRE_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const long long B = cfg->batch;
  fire_status_t e = fire_mlp_reserve(m, B);
  if (e != FIRE_OK) return e;
  if (!m->have_stats) {
    // input statistics from one synthetic batch of the same distribution
    MCK(launch_mlp_synth(m->ctx_t, m->ctx_c, B, -1 - B, cfg->seed, cfg->pfire, cfg->noise_rel,
                         cfg->noise_abs, nullptr, nullptr, m->Din, m->x, nullptr, nullptr, nullptr,
                         m->rad, st));
    MCK(launch_colstats(m->rad, B, m->ctx_t.nb, m->mean, m->istd, st));
    m->have_stats = 1;
  }
  for (long long s = 0; s < cfg->steps; s++) {
    const long long sample0 = cfg->sample0 + s * B;
    MCK(launch_mlp_synth(m->ctx_t, m->ctx_c, B, sample0, cfg->seed, cfg->pfire, cfg->noise_rel,
                         cfg->noise_abs, m->mean, m->istd, m->Din, m->x, m->xT, m->tgt, m->msk,
                         nullptr, st));
    e = forward_rows(m, B, true, st);
    if (e != FIRE_OK) return e;
    e = backward_rows(m, B, st);
    if (e != FIRE_OK) return e;
    const int t = (int)(++m->step);
    MCK(launch_adam(m->W1, m->gW1, 0, m->mW1, m->vW1, m->H, m->Din, cfg->lr, t, m->W1b, m->W1T, st));
    MCK(launch_adam(m->b1, m->gb1, 0, m->mb1, m->vb1, 1, m->H, cfg->lr, t, nullptr, nullptr, st));
    MCK(launch_adam(m->W2, m->gW2, 0, m->mW2, m->vW2, m->H, m->H, cfg->lr, t, m->W2b, m->W2T, st));
    MCK(launch_adam(m->b2, m->gb2, 0, m->mb2, m->vb2, 1, m->H, cfg->lr, t, nullptr, nullptr, st));
    MCK(launch_adam(m->W3, m->gW3T, 1, m->mW3, m->vW3, 16, m->H, cfg->lr, t, m->W3b, m->W3T, st));
    MCK(launch_adam(m->b3, m->gb3, 0, m->mb3, m->vb3, 1, 16, cfg->lr, t, nullptr, nullptr, st));
    if (loss_host) MCK(cudaMemcpyAsync(loss_host + s, m->loss, 4, cudaMemcpyDeviceToHost, st));
  }
  m->sample_next = cfg->sample0 + cfg->steps * B;
  if (loss_host) MCK(cudaStreamSynchronize(st));
  return FIRE_OK;
}

fire_status_t fire_mlp_infer(fire_mlp_t *m, const float *radiance, int64_t n, float *z_out,
                             float *init_out, fire_stream_t stream) {
  if (!m || n < 0 || (n && !radiance)) return FIRE_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const long long chunk = 1 << 17;
  fire_status_t e = fire_mlp_reserve(m, n < chunk ? (n + 127) / 128 * 128 : chunk);
  if (e != FIRE_OK) return e;
  for (long long i0 = 0; i0 < n; i0 += chunk) {
    const long long b = n - i0 < chunk ? n - i0 : chunk;
    MCK(launch_mlp_input(radiance + i0 * m->ctx_t.nb, b, m->ctx_t.nb, m->Din, m->mean, m->istd, m->x,
                         nullptr, 0, st));
    e = forward_rows(m, b, false, st);
    if (e != FIRE_OK) return e;
    if (z_out) MCK(cudaMemcpyAsync(z_out + i0 * 16, m->z, b * 16 * 4, cudaMemcpyDeviceToDevice, st));
    if (init_out) MCK(launch_mlp_to_init(m->z, b, m->K, m->ctx_c, init_out + i0 * (m->K + 8), st));
  }
  return FIRE_OK;
}

fire_status_t fire_mlp_gradients(fire_mlp_t *m, const float *x, const float *tgt, const float *msk,
                                 int64_t B, float *grads, float *loss, fire_stream_t stream) {
  if (!m || !x || !tgt || !msk || !grads || B < 1) return FIRE_ERR_ARG;
  if (B & 7) return FIRE_ERR_SHAPE;   // B is a GEMM K dimension: 16-byte rows
  cudaStream_t st = (cudaStream_t)stream;
  fire_status_t e = fire_mlp_reserve(m, (B + 127) / 128 * 128);
  if (e != FIRE_OK) return e;
  // x is already standardised (fp32 [B][Din]): identity statistics for the copy
  float *ones = nullptr, *zeros = nullptr;
  MCK(dalloc(&ones, m->Din));
  MCK(dalloc(&zeros, m->Din));
  {
    float *h = new float[2 * m->Din];
    for (int i = 0; i < m->Din; i++) { h[i] = 0.f; h[m->Din + i] = 1.f; }
    cudaMemcpy(zeros, h, m->Din * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(ones, h + m->Din, m->Din * 4, cudaMemcpyHostToDevice);
    delete[] h;
  }
  MCK(launch_mlp_input(x, B, m->Din, m->Din, zeros, ones, m->x, m->xT, B, st));
  MCK(cudaMemcpyAsync(m->tgt, tgt, B * 16 * 4, cudaMemcpyDeviceToDevice, st));
  MCK(cudaMemcpyAsync(m->msk, msk, B * 16 * 4, cudaMemcpyDeviceToDevice, st));
  e = forward_rows(m, B, true, st);
  if (e == FIRE_OK) e = backward_rows(m, B, st);
  if (e == FIRE_OK) {
    const size_t H = m->H, D = m->Din;
    float *p = grads;
    cudaMemcpyAsync(p, m->gW1, H * D * 4, cudaMemcpyDeviceToDevice, st); p += H * D;
    cudaMemcpyAsync(p, m->gb1, H * 4, cudaMemcpyDeviceToDevice, st); p += H;
    cudaMemcpyAsync(p, m->gW2, H * H * 4, cudaMemcpyDeviceToDevice, st); p += H * H;
    cudaMemcpyAsync(p, m->gb2, H * 4, cudaMemcpyDeviceToDevice, st); p += H;
    cudaMemcpyAsync(p, m->gW3T, H * 16 * 4, cudaMemcpyDeviceToDevice, st); p += H * 16;
    cudaMemcpyAsync(p, m->gb3, 16 * 4, cudaMemcpyDeviceToDevice, st);
    if (loss) cudaMemcpyAsync(loss, m->loss, 4, cudaMemcpyDeviceToDevice, st);
  }
  cudaStreamSynchronize(st);
  dev_free(ones);
  dev_free(zeros);
  return e;
}

int64_t fire_mlp_param_count(const fire_mlp_t *m) {
  if (!m) return 0;
  return (int64_t)m->H * m->Din + m->H + (int64_t)m->H * m->H + m->H + 16LL * m->H + 16 + 2LL * m->Din;
}

fire_status_t fire_mlp_params(fire_mlp_t *m, float *get, const float *set) {
  if (!m) return FIRE_ERR_ARG;
  const size_t H = m->H, D = m->Din;
  float *dev[] = {m->W1, m->b1, m->W2, m->b2, m->W3, m->b3, m->mean, m->istd};
  size_t cnt[] = {H * D, H, H * H, H, 16 * H, 16, D, D};
  size_t off = 0;
  for (int i = 0; i < 8; i++) {
    if (get) MCK(cudaMemcpy(get + off, dev[i], cnt[i] * 4, cudaMemcpyDeviceToHost));
    if (set) MCK(cudaMemcpy(dev[i], set + off, cnt[i] * 4, cudaMemcpyHostToDevice));
    off += cnt[i];
  }
  if (set) {
    m->have_stats = 1;
    fire_status_t e = refresh_bf16(m, 0);
    if (e != FIRE_OK) return e;
    MCK(cudaDeviceSynchronize());
  }
  return FIRE_OK;
}

// checkpoint: magic, shape, step and sample counters, parameters, Adam
// moments, FNV-1a 64 checksum of everything before it
fire_status_t fire_mlp_save(fire_mlp_t *m, const char *path) {
  if (!m || !path) return FIRE_ERR_ARG;
  const size_t H = m->H, D = m->Din;
  float *dev[] = {m->W1, m->b1, m->W2, m->b2, m->W3, m->b3, m->mean, m->istd, m->mW1, m->vW1,
                  m->mb1, m->vb1, m->mW2, m->vW2, m->mb2, m->vb2, m->mW3, m->vW3, m->mb3, m->vb3};
  size_t cnt[] = {H * D, H, H * H, H, 16 * H, 16, D, D, H * D, H * D, H, H, H * H, H * H, H, H,
                  16 * H, 16 * H, 16, 16};
  size_t total = 0;
  for (size_t c : cnt) total += c;
  float *buf = new (std::nothrow) float[total];
  if (!buf) return FIRE_ERR_NOMEM;
  size_t off = 0;
  for (int i = 0; i < 20; i++) {
    if (cudaMemcpy(buf + off, dev[i], cnt[i] * 4, cudaMemcpyDeviceToHost) != cudaSuccess) {
      delete[] buf;
      return FIRE_ERR_CUDA;
    }
    off += cnt[i];
  }
  int64_t hdr[8] = {0x31504C4D45524946LL /* "FIREMLP1" */, 1, m->K, m->ctx_t.nb, m->Din, m->H,
                    m->step, m->sample_next};
  int64_t flags = m->have_stats;
  uint64_t h = fnv1a(hdr, sizeof(hdr), 1469598103934665603ull);
  h = fnv1a(&flags, sizeof(flags), h);
  h = fnv1a(buf, total * 4, h);
  FILE *f = fopen(path, "wb");
  fire_status_t st = FIRE_OK;
  if (!f) st = FIRE_ERR_CHECKPOINT;
  else {
    if (fwrite(hdr, sizeof(hdr), 1, f) != 1 || fwrite(&flags, sizeof(flags), 1, f) != 1 ||
        fwrite(buf, 4, total, f) != total || fwrite(&h, sizeof(h), 1, f) != 1)
      st = FIRE_ERR_CHECKPOINT;
    fclose(f);
  }
  delete[] buf;
  return st;
}

fire_status_t fire_mlp_load(fire_mlp_t *m, const char *path) {
  if (!m || !path) return FIRE_ERR_ARG;
  const size_t H = m->H, D = m->Din;
  float *dev[] = {m->W1, m->b1, m->W2, m->b2, m->W3, m->b3, m->mean, m->istd, m->mW1, m->vW1,
                  m->mb1, m->vb1, m->mW2, m->vW2, m->mb2, m->vb2, m->mW3, m->vW3, m->mb3, m->vb3};
  size_t cnt[] = {H * D, H, H * H, H, 16 * H, 16, D, D, H * D, H * D, H, H, H * H, H * H, H, H,
                  16 * H, 16 * H, 16, 16};
  size_t total = 0;
  for (size_t c : cnt) total += c;
  FILE *f = fopen(path, "rb");
  if (!f) return FIRE_ERR_CHECKPOINT;
  int64_t hdr[8], flags = 0;
  uint64_t h_file = 0;
  float *buf = new (std::nothrow) float[total];
  fire_status_t st = FIRE_OK;
  if (!buf) st = FIRE_ERR_NOMEM;
  else if (fread(hdr, sizeof(hdr), 1, f) != 1 || fread(&flags, sizeof(flags), 1, f) != 1 ||
           fread(buf, 4, total, f) != total || fread(&h_file, sizeof(h_file), 1, f) != 1)
    st = FIRE_ERR_CHECKPOINT;
  fclose(f);
  if (st == FIRE_OK) {
    uint64_t h = fnv1a(hdr, sizeof(hdr), 1469598103934665603ull);
    h = fnv1a(&flags, sizeof(flags), h);
    h = fnv1a(buf, total * 4, h);
    if (h != h_file || hdr[0] != 0x31504C4D45524946LL || hdr[1] != 1 || hdr[2] != m->K ||
        hdr[3] != m->ctx_t.nb || hdr[4] != m->Din || hdr[5] != m->H)
      st = FIRE_ERR_CHECKPOINT;
  }
  if (st == FIRE_OK) {
    size_t off = 0;
    for (int i = 0; i < 20 && st == FIRE_OK; i++) {
      if (cudaMemcpy(dev[i], buf + off, cnt[i] * 4, cudaMemcpyHostToDevice) != cudaSuccess)
        st = FIRE_ERR_CUDA;
      off += cnt[i];
    }
    m->step = hdr[6];
    m->sample_next = hdr[7];
    m->have_stats = (int)flags;
    if (st == FIRE_OK) st = refresh_bf16(m, 0);
    if (st == FIRE_OK && cudaDeviceSynchronize() != cudaSuccess) st = FIRE_ERR_CUDA;
  }
  delete[] buf;
  return st;
}

int64_t fire_mlp_next_sample(const fire_mlp_t *m) { return m ? m->sample_next : 0; }

}  // extern "C"
