// Selector features of one traversal level, shared by the fused decision
// kernel and the batched engine (each translation unit inlines its own copy).
#pragma once

#include <stdint.h>

namespace gi {

// features of one level (same definition as the selector's training data)
__device__ __forceinline__ void level_features(float *x, int64_t n, int64_t m, int32_t maxdeg, int64_t nf, int64_t mf, int64_t nu,
                               int64_t mu, int32_t level, int32_t was_pull, int64_t nf_prev) {
  float V = (float)(n > 0 ? n : 1), E = (float)(m > 0 ? m : 1);
  x[0] = log2f(1.0f + (float)nf);
  x[1] = log2f(1.0f + (float)mf);
  x[2] = log2f(1.0f + (float)nu);
  x[3] = log2f(1.0f + (float)mu);
  x[4] = log2f(1.0f + (float)n);
  x[5] = log2f(1.0f + (float)m);
  x[6] = (float)nf / V;
  x[7] = (float)mf / E;
  x[8] = (float)nu / V;
  x[9] = (float)mu / E;
  x[10] = log2f(1.0f + (float)((double)mf / (double)(nf > 0 ? nf : 1)));
  x[11] = log2f(1.0f + (float)maxdeg);
  x[12] = log2f(1.0f + (float)((double)m / (double)V));
  x[13] = log2f(1.0f + (float)level);
  x[14] = was_pull ? 1.0f : 0.0f;
  x[15] = log2f(1.0f + (float)nf_prev);
}

}  // namespace gi
