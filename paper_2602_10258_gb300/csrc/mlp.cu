// Training of the beam / stop network of the learned search policy: forward
// pass, back-propagation and Adam, all on the GPU.
//
// Network: 12 features -> 64 ReLU -> 64 ReLU -> nl + 1 outputs (nl logits
// over the beam ladder, one stop-hop output).  Loss of a batch of B rows:
// mean cross-entropy of the logits against the beam class plus lam * mean
// squared error of the stop output against its target.
//
// K_mlp1 (mlp_grad_kernel): one CTA per 64-row slice of the batch.  The
//   slice's activations stay in shared memory; the CTA writes its partial
//   gradient (every parameter summed over its rows, rows in order) and its
//   partial loss.
// K_mlp2 (mlp_reduce_kernel): one thread per parameter sums the partials over
//   the slices in order (so the result does not depend on scheduling) and,
//   when training, applies the Adam update to that parameter.
//
// The network is a few thousand parameters and trains offline, so the
// kernels favour a fixed summation order over throughput.
#include <cmath>
#include <vector>

#include "launch.h"

namespace jag {

constexpr int kMlpRows = 64;      // rows per CTA of K_mlp1
constexpr int kMlpThreads = 256;
constexpr int kF = JAG_MLP_FEATURES, kH = JAG_MLP_HIDDEN;

__host__ __device__ inline int64_t mlp_params(int nl) {
  return (int64_t)kH * kF + kH + kH * kH + kH + (int64_t)(nl + 1) * kH + (nl + 1);
}

// Shared-memory layout of K_mlp1 (floats).
struct MlpSmem {
  float *x, *a1, *a2, *z, *d1, *d2, *w2, *w3, *rl;
  int32_t *y;
  float *t;
};

__host__ __device__ inline size_t mlp_smem_floats(int nl) {
  const int no = nl + 1;
  return (size_t)kMlpRows * kF + 4 * (size_t)kMlpRows * kH + (size_t)kMlpRows * no + (size_t)kH * kH +
         (size_t)no * kH + 3 * kMlpRows;
}

__global__ void __launch_bounds__(kMlpThreads)
mlp_grad_kernel(int nl, const float *__restrict__ params, const float *__restrict__ X,
                const int32_t *__restrict__ Y, const float *__restrict__ T, int64_t row0, int64_t B, float lam,
                float *__restrict__ part, float *__restrict__ lpart) {
  extern __shared__ __align__(16) float sm[];
  const int no = nl + 1, tid = threadIdx.x;
  const int64_t P = mlp_params(nl);
  const float *W1 = params, *b1 = W1 + kH * kF, *W2 = b1 + kH, *b2 = W2 + kH * kH, *W3 = b2 + kH,
              *b3 = W3 + no * kH;
  MlpSmem s;
  s.x = sm;
  s.a1 = s.x + kMlpRows * kF;
  s.a2 = s.a1 + kMlpRows * kH;
  s.d1 = s.a2 + kMlpRows * kH;
  s.d2 = s.d1 + kMlpRows * kH;
  s.z = s.d2 + kMlpRows * kH;
  s.w2 = s.z + kMlpRows * no;
  s.w3 = s.w2 + kH * kH;
  s.rl = s.w3 + no * kH;
  s.t = s.rl + kMlpRows;
  s.y = reinterpret_cast<int32_t *>(s.t + kMlpRows);
  const int64_t r0 = (int64_t)blockIdx.x * kMlpRows;
  const int rows = (int)min64(kMlpRows, B - r0);
  const float inv_b = 1.f / (float)B;
  for (int i = tid; i < rows * kF; i += kMlpThreads) s.x[i] = X[(row0 + r0) * kF + i];
  for (int i = tid; i < kH * kH; i += kMlpThreads) s.w2[i] = W2[i];
  for (int i = tid; i < no * kH; i += kMlpThreads) s.w3[i] = W3[i];
  for (int r = tid; r < rows; r += kMlpThreads) { s.y[r] = Y[row0 + r0 + r]; s.t[r] = T[row0 + r0 + r]; }
  __syncthreads();
  // forward
  for (int e = tid; e < rows * kH; e += kMlpThreads) {
    const int r = e / kH, j = e % kH;
    float acc = b1[j];
    for (int i = 0; i < kF; ++i) acc = fmaf(W1[j * kF + i], s.x[r * kF + i], acc);
    s.a1[e] = acc;
  }
  __syncthreads();
  for (int e = tid; e < rows * kH; e += kMlpThreads) {
    const int r = e / kH, j = e % kH;
    float acc = b2[j];
    for (int i = 0; i < kH; ++i) acc = fmaf(s.w2[j * kH + i], fmaxf(s.a1[r * kH + i], 0.f), acc);
    s.a2[e] = acc;
  }
  __syncthreads();
  for (int e = tid; e < rows * no; e += kMlpThreads) {
    const int r = e / no, o = e % no;
    float acc = b3[o];
    for (int i = 0; i < kH; ++i) acc = fmaf(s.w3[o * kH + i], fmaxf(s.a2[r * kH + i], 0.f), acc);
    s.z[e] = acc;
  }
  __syncthreads();
  // loss of each row and d loss / d z (in place of z)
  for (int r = tid; r < rows; r += kMlpThreads) {
    float *z = s.z + r * no;
    const int y = s.y[r];
    float mx = z[0];
    for (int o = 1; o < nl; ++o) mx = fmaxf(mx, z[o]);
    float se = 0.f;
    for (int o = 0; o < nl; ++o) se += expf(z[o] - mx);
    const float lse = mx + logf(se);
    const bool yok = y >= 0 && y < nl;
    const float dz = z[nl] - s.t[r];
    s.rl[r] = (yok ? lse - z[y] : NAN) + lam * dz * dz;
    for (int o = 0; o < nl; ++o) z[o] = (expf(z[o] - mx) / se - (o == y ? 1.f : 0.f)) * inv_b;
    z[nl] = 2.f * lam * dz * inv_b;
  }
  __syncthreads();
  // d loss / d a2 and d loss / d a1
  for (int e = tid; e < rows * kH; e += kMlpThreads) {
    const int r = e / kH, j = e % kH;
    float acc = 0.f;
    for (int o = 0; o < no; ++o) acc = fmaf(s.z[r * no + o], s.w3[o * kH + j], acc);
    s.d2[e] = s.a2[e] > 0.f ? acc : 0.f;
  }
  __syncthreads();
  for (int e = tid; e < rows * kH; e += kMlpThreads) {
    const int r = e / kH, i = e % kH;
    float acc = 0.f;
    for (int j = 0; j < kH; ++j) acc = fmaf(s.d2[r * kH + j], s.w2[j * kH + i], acc);
    s.d1[e] = s.a1[e] > 0.f ? acc : 0.f;
  }
  __syncthreads();
  // partial gradient of every parameter over this slice's rows, in order
  float *out = part + (int64_t)blockIdx.x * P;
  for (int64_t p = tid; p < P; p += kMlpThreads) {
    float acc = 0.f;
    int64_t q = p;
    if (q < kH * kF) {
      const int j = (int)(q / kF), i = (int)(q % kF);
      for (int r = 0; r < rows; ++r) acc = fmaf(s.d1[r * kH + j], s.x[r * kF + i], acc);
    } else if ((q -= kH * kF) < kH) {
      for (int r = 0; r < rows; ++r) acc += s.d1[r * kH + q];
    } else if ((q -= kH) < kH * kH) {
      const int j = (int)(q / kH), i = (int)(q % kH);
      for (int r = 0; r < rows; ++r) acc = fmaf(s.d2[r * kH + j], fmaxf(s.a1[r * kH + i], 0.f), acc);
    } else if ((q -= kH * kH) < kH) {
      for (int r = 0; r < rows; ++r) acc += s.d2[r * kH + q];
    } else if ((q -= kH) < no * kH) {
      const int o = (int)(q / kH), i = (int)(q % kH);
      for (int r = 0; r < rows; ++r) acc = fmaf(s.z[r * no + o], fmaxf(s.a2[r * kH + i], 0.f), acc);
    } else {
      q -= no * kH;
      for (int r = 0; r < rows; ++r) acc += s.z[r * no + q];
    }
    out[p] = acc;
  }
  if (tid == 0) {
    float l = 0.f;
    for (int r = 0; r < rows; ++r) l += s.rl[r];
    lpart[blockIdx.x] = l;
  }
}

// Sum of the slices' partials in slice order; with adam != 0 the Adam step
// theta -= lr * (m c1) / (sqrt(v c2) + eps) follows (c1, c2: the bias
// corrections 1 / (1 - beta^t)).
__global__ void __launch_bounds__(256)
mlp_reduce_kernel(int64_t P, int nslices, const float *__restrict__ part, const float *__restrict__ lpart,
                  int64_t B, float *grad, float *loss, float *loss_acc, int adam, float *params, float *am,
                  float *av, float lr, float c1, float c2) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p == 0) {
    float l = 0.f;
    for (int b = 0; b < nslices; ++b) l += lpart[b];
    l /= (float)B;
    if (loss) *loss = l;
    if (loss_acc) *loss_acc += l;
  }
  if (p >= P) return;
  float g = 0.f;
  for (int b = 0; b < nslices; ++b) g += part[(int64_t)b * P + p];
  if (grad) grad[p] = g;
  if (adam) {
    const float m = 0.9f * am[p] + 0.1f * g;
    const float v = 0.999f * av[p] + 0.001f * g * g;
    am[p] = m;
    av[p] = v;
    params[p] -= lr * (m * c1) / (sqrtf(v * c2) + 1e-8f);
  }
}

__global__ void mlp_export_kernel(int64_t nw, int nl, const float *params, uint16_t *w, float *b) {
  const int no = nl + 1;
  const int64_t n1 = (int64_t)kH * kF, n2 = (int64_t)kH * kH;
  const int64_t nb = 2 * kH + no;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nw + nb; i += (int64_t)gridDim.x * blockDim.x) {
    if (i < nw) {
      // weight i of W1 | W2 | W3 -> its place in the flat parameter vector
      const int64_t src = i < n1 ? i : i < n1 + n2 ? i + kH : i + 2 * kH;
      w[i] = __bfloat16_as_ushort(__float2bfloat16_rn(params[src]));
    } else {
      const int64_t j = i - nw;
      const int64_t src = j < kH ? n1 + j : j < 2 * kH ? n1 + kH + n2 + (j - kH) : n1 + 2 * kH + n2 + no * kH + (j - 2 * kH);
      b[j] = params[src];
    }
  }
}

// One batch (rows [row0, row0 + B)): partials then reduction.
static cudaError_t mlp_batch(int nl, const float *params, const float *X, const int32_t *y, const float *t,
                             int64_t row0, int64_t B, float lam, float *part, float *lpart, float *grad,
                             float *loss, float *loss_acc, int adam, float *am, float *av, float lr, float c1,
                             float c2, cudaStream_t st) {
  const int64_t P = mlp_params(nl);
  const int ns = (int)((B + kMlpRows - 1) / kMlpRows);
  const size_t smem = mlp_smem_floats(nl) * sizeof(float);
  mlp_grad_kernel<<<ns, kMlpThreads, smem, st>>>(nl, params, X, y, t, row0, B, lam, part, lpart);
  mlp_reduce_kernel<<<(unsigned)((P + 255) / 256), 256, 0, st>>>(P, ns, part, lpart, B, grad, loss, loss_acc, adam,
                                                                 const_cast<float *>(params), am, av, lr, c1, c2);
  return cudaGetLastError();
}

static jag_status mlp_setup(int nl) {
  const size_t smem = mlp_smem_floats(nl) * sizeof(float);
  if (cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return set_error(JAG_ECUDA, "cannot reserve shared memory for the network kernels");
  return JAG_OK;
}

}  // namespace jag

using namespace jag;

extern "C" JAG_API jag_status jag_mlp_loss_grad(int32_t n_ladder, const float *params, const float *X,
                                                const int32_t *y, const float *t, int64_t m, float lam,
                                                float *grad, float *loss, void *stream) {
  if (n_ladder < 1 || n_ladder > 16) return set_error(JAG_EINVAL, "n_ladder must be in [1, 16]");
  if (!params || !X || !y || !t || !grad || !loss) return set_error(JAG_EINVAL, "NULL argument");
  if (m < 1) return set_error(JAG_EINVAL, "m must be >= 1");
  if (!(lam >= 0.f) || !std::isfinite(lam)) return set_error(JAG_EINVAL, "lam must be finite and >= 0");
  if (jag_status s = mlp_setup(n_ladder)) return s;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t P = mlp_params(n_ladder);
  const int64_t ns = (m + kMlpRows - 1) / kMlpRows;
  float *buf = nullptr;
  if (cudaMallocAsync((void **)&buf, (size_t)(ns * P + ns) * sizeof(float), st) != cudaSuccess)
    return set_error(JAG_ENOMEM, "cannot allocate the gradient partials");
  cudaError_t e = mlp_batch(n_ladder, params, X, y, t, 0, m, lam, buf, buf + ns * P, grad, loss, nullptr, 0,
                            nullptr, nullptr, 0.f, 0.f, 0.f, st);
  cudaFreeAsync(buf, st);
  if (e != cudaSuccess) return set_error(JAG_ECUDA, cudaGetErrorString(e));
  return JAG_OK;
}

extern "C" JAG_API jag_status jag_mlp_train(int32_t n_ladder, float *params, float *adam_m, float *adam_v,
                                            int64_t *adam_step, const float *X, const int32_t *y, const float *t,
                                            int64_t m, int32_t epochs, int32_t batch, float lr, float lam,
                                            float *loss_trace, void *stream) {
  if (n_ladder < 1 || n_ladder > 16) return set_error(JAG_EINVAL, "n_ladder must be in [1, 16]");
  if (!params || !adam_m || !adam_v || !adam_step || !X || !y || !t) return set_error(JAG_EINVAL, "NULL argument");
  if (m < 1 || epochs < 0 || batch < 1) return set_error(JAG_EINVAL, "m, batch must be >= 1 and epochs >= 0");
  if (!(lam >= 0.f) || !std::isfinite(lam) || !(lr > 0.f) || !std::isfinite(lr))
    return set_error(JAG_EINVAL, "lr must be > 0 and lam >= 0, both finite");
  if (*adam_step < 0) return set_error(JAG_EINVAL, "adam_step must be >= 0");
  if (jag_status s = mlp_setup(n_ladder)) return s;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t P = mlp_params(n_ladder);
  const int64_t B = batch < m ? batch : m;
  const int64_t ns = (B + kMlpRows - 1) / kMlpRows;
  const int64_t nb = (m + B - 1) / B;
  float *buf = nullptr;
  const size_t nbuf = (size_t)(ns * P + ns + (epochs > 0 ? epochs : 1));
  if (cudaMallocAsync((void **)&buf, nbuf * sizeof(float), st) != cudaSuccess)
    return set_error(JAG_ENOMEM, "cannot allocate the training scratch");
  float *part = buf, *lpart = buf + ns * P, *acc = lpart + ns;
  cudaError_t e = cudaMemsetAsync(acc, 0, sizeof(float) * (size_t)(epochs > 0 ? epochs : 1), st);
  int64_t step = *adam_step;
  for (int ep = 0; ep < epochs && e == cudaSuccess; ++ep) {
    for (int64_t b = 0; b < nb && e == cudaSuccess; ++b) {
      const int64_t row0 = b * B, rows = row0 + B <= m ? B : m - row0;
      ++step;
      const float c1 = (float)(1.0 / (1.0 - std::pow(0.9, (double)step)));
      const float c2 = (float)(1.0 / (1.0 - std::pow(0.999, (double)step)));
      e = mlp_batch(n_ladder, params, X, y, t, row0, rows, lam, part, lpart, nullptr, nullptr, acc + ep, 1, adam_m,
                    adam_v, lr, c1, c2, st);
    }
  }
  std::vector<float> tr((size_t)(epochs > 0 ? epochs : 1));
  if (e == cudaSuccess && loss_trace && epochs > 0)
    e = cudaMemcpyAsync(tr.data(), acc, sizeof(float) * (size_t)epochs, cudaMemcpyDeviceToHost, st);
  cudaFreeAsync(buf, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return set_error(JAG_ECUDA, cudaGetErrorString(e));
  if (loss_trace)
    for (int ep = 0; ep < epochs; ++ep) loss_trace[ep] = tr[(size_t)ep] / (float)nb;
  *adam_step = step;
  return JAG_OK;
}

extern "C" JAG_API jag_status jag_mlp_export(int32_t n_ladder, const float *params, uint16_t *w_bf16, float *b_f32,
                                             void *stream) {
  if (n_ladder < 1 || n_ladder > 16) return set_error(JAG_EINVAL, "n_ladder must be in [1, 16]");
  if (!params || !w_bf16 || !b_f32) return set_error(JAG_EINVAL, "NULL argument");
  const int64_t nw = (int64_t)kH * kF + (int64_t)kH * kH + (int64_t)(n_ladder + 1) * kH;
  mlp_export_kernel<<<32, 256, 0, (cudaStream_t)stream>>>(nw, n_ladder, params, w_bf16, b_f32);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(JAG_ECUDA, cudaGetErrorString(e));
  return JAG_OK;
}
