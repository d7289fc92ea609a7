/*
 * FP64 reference of the learned SGS closure network and its training step.
 * The paper has no learned closure; this network (13 -> 64 -> 64 -> 2, SiLU)
 * is an extension of the method.  The oracle only provides the plain
 * definitions so that the GPU BF16 forward/backward kernels can be checked:
 *   h1 = silu(W1 x + b1), h2 = silu(W2 h1 + b2), y = W3 h2 + b3,
 *   silu(a) = a sigma(a), silu'(a) = sigma(a) (1 + a (1 - sigma(a))),
 *   loss = 1/(2n) sum_samples |y - t|^2, Adam of Kingma & Ba (2015).
 * Test infrastructure only (see oracle.h).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include "oracle.h"

static double sigmoid(double a) { return 1.0 / (1.0 + exp(-a)); }

void orc_mlp_forward(int n, const double *X, const double *W1, const double *b1, const double *W2,
                     const double *b2, const double *W3, const double *b3, double *Y) {
  for (int s = 0; s < n; ++s) {
    double h1[64], h2[64];
    for (int o = 0; o < 64; ++o) {
      double a = b1[o];
      for (int i = 0; i < 13; ++i) a += W1[o * 13 + i] * X[s * 13 + i];
      h1[o] = a * sigmoid(a);
    }
    for (int o = 0; o < 64; ++o) {
      double a = b2[o];
      for (int i = 0; i < 64; ++i) a += W2[o * 64 + i] * h1[i];
      h2[o] = a * sigmoid(a);
    }
    for (int o = 0; o < 2; ++o) {
      double a = b3[o];
      for (int i = 0; i < 64; ++i) a += W3[o * 64 + i] * h2[i];
      Y[s * 2 + o] = a;
    }
  }
}

/* BF16 (8-bit significand) value of x: x rounded to FP32, then to BF16 with
 * round-to-nearest-even on the 16 dropped bits. */
double orc_bf16(double x) {
  union { float f; uint32_t u; } v;
  v.f = (float)x;
  uint32_t lsb = (v.u >> 16) & 1u;
  v.u = (v.u + 0x7FFFu + lsb) & 0xFFFF0000u;
  return (double)v.f;
}

/* The closure network as the learned closure defines it: inputs and hidden
 * activations stored in BF16, weights given (BF16 values), biases and the
 * sums exact. */
void orc_mlp_forward_bf16(int n, const double *X, const double *W1, const double *b1, const double *W2,
                          const double *b2, const double *W3, const double *b3, double *Y) {
  for (int s = 0; s < n; ++s) {
    double x[13], h1[64], h2[64];
    for (int i = 0; i < 13; ++i) x[i] = orc_bf16(X[s * 13 + i]);
    for (int o = 0; o < 64; ++o) {
      double a = b1[o];
      for (int i = 0; i < 13; ++i) a += W1[o * 13 + i] * x[i];
      h1[o] = orc_bf16(a * sigmoid(a));
    }
    for (int o = 0; o < 64; ++o) {
      double a = b2[o];
      for (int i = 0; i < 64; ++i) a += W2[o * 64 + i] * h1[i];
      h2[o] = orc_bf16(a * sigmoid(a));
    }
    for (int o = 0; o < 2; ++o) {
      double a = b3[o];
      for (int i = 0; i < 64; ++i) a += W3[o * 64 + i] * h2[i];
      Y[s * 2 + o] = a;
    }
  }
}

double orc_mlp_loss_grad(int n, const double *X, const double *T, const double *W1, const double *b1,
                         const double *W2, const double *b2, const double *W3, const double *b3, double *gW1,
                         double *gb1, double *gW2, double *gb2, double *gW3, double *gb3) {
  for (int k = 0; k < 64 * 13; ++k) gW1[k] = 0.0;
  for (int k = 0; k < 64 * 64; ++k) gW2[k] = 0.0;
  for (int k = 0; k < 2 * 64; ++k) gW3[k] = 0.0;
  for (int k = 0; k < 64; ++k) gb1[k] = gb2[k] = 0.0;
  gb3[0] = gb3[1] = 0.0;
  double loss = 0.0;
  for (int s = 0; s < n; ++s) {
    const double *x = X + s * 13;
    double a1[64], h1[64], a2[64], h2[64], y[2];
    for (int o = 0; o < 64; ++o) {
      double a = b1[o];
      for (int i = 0; i < 13; ++i) a += W1[o * 13 + i] * x[i];
      a1[o] = a;
      h1[o] = a * sigmoid(a);
    }
    for (int o = 0; o < 64; ++o) {
      double a = b2[o];
      for (int i = 0; i < 64; ++i) a += W2[o * 64 + i] * h1[i];
      a2[o] = a;
      h2[o] = a * sigmoid(a);
    }
    for (int o = 0; o < 2; ++o) {
      double a = b3[o];
      for (int i = 0; i < 64; ++i) a += W3[o * 64 + i] * h2[i];
      y[o] = a;
    }
    /* backward: dL/dy = (y - t)/n */
    double dy[2];
    for (int o = 0; o < 2; ++o) {
      double r = y[o] - T[s * 2 + o];
      loss += 0.5 * r * r / n;
      dy[o] = r / n;
    }
    double dh2[64], da2[64], dh1[64], da1[64];
    for (int i = 0; i < 64; ++i) {
      double acc = 0.0;
      for (int o = 0; o < 2; ++o) {
        gW3[o * 64 + i] += dy[o] * h2[i];
        acc += W3[o * 64 + i] * dy[o];
      }
      dh2[i] = acc;
    }
    for (int o = 0; o < 2; ++o) gb3[o] += dy[o];
    for (int i = 0; i < 64; ++i) {
      double sg = sigmoid(a2[i]);
      da2[i] = dh2[i] * sg * (1.0 + a2[i] * (1.0 - sg));
    }
    for (int i = 0; i < 64; ++i) {
      double acc = 0.0;
      for (int o = 0; o < 64; ++o) {
        gW2[o * 64 + i] += da2[o] * h1[i];
        acc += W2[o * 64 + i] * da2[o];
      }
      dh1[i] = acc;
    }
    for (int o = 0; o < 64; ++o) gb2[o] += da2[o];
    for (int i = 0; i < 64; ++i) {
      double sg = sigmoid(a1[i]);
      da1[i] = dh1[i] * sg * (1.0 + a1[i] * (1.0 - sg));
    }
    for (int o = 0; o < 64; ++o) {
      for (int i = 0; i < 13; ++i) gW1[o * 13 + i] += da1[o] * x[i];
      gb1[o] += da1[o];
    }
  }
  return loss;
}

void orc_adam(int n, double *theta, const double *g, double *m, double *v, int t, double lr, double beta1,
              double beta2, double eps) {
  double c1 = 1.0 - pow(beta1, t), c2 = 1.0 - pow(beta2, t);
  for (int k = 0; k < n; ++k) {
    m[k] = beta1 * m[k] + (1.0 - beta1) * g[k];
    v[k] = beta2 * v[k] + (1.0 - beta2) * g[k] * g[k];
    double mh = m[k] / c1, vh = v[k] / c2;
    theta[k] -= lr * mh / (sqrt(vh) + eps);
  }
}
