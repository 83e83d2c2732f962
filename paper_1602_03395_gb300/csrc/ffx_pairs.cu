// Positive-P pairs (Sec. 7, Generalizations): the two fields psi and psi+
// evolve by the map T and by its complex conjugate.  conj(T) psi+ is computed
// as conj(T conj(psi+)), so both fields run through the same passes:
//   conj_copy_kernel:     W2 = conj(psi+)
//   (the forward map on psi -> W1 and on W2 -> W2)
//   pair_density_kernel:  rho = Re(Psibar+ Psibar) = Re(conj(W2) W1), per
//                         realization or summed over the batch in order.
#include "ffx_internal.h"

namespace ffx {

namespace {

__global__ void conj_copy_kernel(const float2* __restrict__ in, float2* __restrict__ out, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float2 v = in[i];
    out[i] = make_float2(v.x, -v.y);
  }
}

__global__ void pair_density_kernel(const float2* __restrict__ w1, const float2* __restrict__ w2, int64_t M,
                                    int64_t batch, int acc, float* __restrict__ out) {
  const int64_t n = acc ? M : M * batch;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (acc) {
      float s = 0.f;
      for (int64_t b = 0; b < batch; ++b) {
        const float2 a = w1[b * M + i], c = w2[b * M + i];
        s += a.x * c.x + a.y * c.y;  // Re(conj(c) a)
      }
      out[i] += s;
    } else {
      const float2 a = w1[i], c = w2[i];
      out[i] = a.x * c.x + a.y * c.y;
    }
  }
}

int blocks_for(int64_t n, int sms) {
  int64_t b = (n + 255) / 256;
  if (b > (int64_t)sms * 16) b = (int64_t)sms * 16;
  return b < 1 ? 1 : (int)b;
}

}  // namespace

cudaError_t launch_conj_copy(const float2* in, float2* out, int64_t n, int sms, cudaStream_t s) {
  conj_copy_kernel<<<blocks_for(n, sms), 256, 0, s>>>(in, out, n);
  return cudaGetLastError();
}

cudaError_t launch_pair_density(const float2* w1, const float2* w2, int64_t M, int64_t batch, int acc, float* out,
                                int sms, cudaStream_t s) {
  pair_density_kernel<<<blocks_for(acc ? M : M * batch, sms), 256, 0, s>>>(w1, w2, M, batch, acc, out);
  return cudaGetLastError();
}

}  // namespace ffx
