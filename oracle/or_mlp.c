/*
 * or_mlp.c -- FP64 reference of the weak-coupling predictor network.
 *
 * TEST INFRASTRUCTURE ONLY (see cp_oracle.h).
 *
 * Network: 40 -> 64 -> 64 -> 64 -> 2 with GELU (x Phi(x), erf form) after
 * each hidden layer and a linear output.  Weights are the FP32 master values
 * rounded to bfloat16 (round to nearest, ties to even); biases are FP32.
 * Everything else is FP64: the products, sums, activations and the
 * gradient, which is taken with respect to the rounded weights.
 * Parameter layout: W1[64][40] b1[64] W2[64][64] b2[64] W3[64][64] b3[64]
 * W4[2][64] b4[2], W[out][in] row-major.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#include "cp_oracle.h"

#define IN OR_MLP_IN
#define HID OR_MLP_HIDDEN
#define OUT OR_MLP_OUT

enum {
  OFF_W1 = 0,
  OFF_B1 = OFF_W1 + HID * IN,
  OFF_W2 = OFF_B1 + HID,
  OFF_B2 = OFF_W2 + HID * HID,
  OFF_W3 = OFF_B2 + HID,
  OFF_B3 = OFF_W3 + HID * HID,
  OFF_W4 = OFF_B3 + HID,
  OFF_B4 = OFF_W4 + OUT * HID,
  NPARAM = OFF_B4 + OUT
};

/* bfloat16 is the upper 16 bits of a binary32 word.  Round to nearest, ties
   to even: add 0x7FFF plus the lowest kept bit, then truncate; NaN stays NaN. */
double or_bf16(float w) {
  uint32_t b;
  memcpy(&b, &w, sizeof b);
  if ((b & 0x7F800000u) == 0x7F800000u && (b & 0x007FFFFFu)) return (double)w;
  const uint32_t lsb = (b >> 16) & 1u;
  b = (b + 0x7FFFu + lsb) & 0xFFFF0000u;
  float r;
  memcpy(&r, &b, sizeof r);
  return (double)r;
}

double or_gelu(double x) { return 0.5 * x * (1.0 + erf(x / sqrt(2.0))); }

double or_gelu_grad(double x) {
  const double pi = 3.14159265358979323846;
  return 0.5 * (1.0 + erf(x / sqrt(2.0))) + x * exp(-0.5 * x * x) / sqrt(2.0 * pi);
}

/* The network's weights as doubles (W rounded to bfloat16, b as given). */
static void load(const float* p, double* w) {
  for (int i = 0; i < NPARAM; ++i) {
    const int is_bias = (i >= OFF_B1 && i < OFF_W2) || (i >= OFF_B2 && i < OFF_W3) ||
                        (i >= OFF_B3 && i < OFF_W4) || i >= OFF_B4;
    w[i] = is_bias ? (double)p[i] : or_bf16(p[i]);
  }
}

/* z = W a + b for one layer (W[nout][nin]). */
static void affine(const double* W, const double* b, const double* a, int nin, int nout,
                   double* z) {
  for (int o = 0; o < nout; ++o) {
    double s = b[o];
    for (int k = 0; k < nin; ++k) s += W[o * nin + k] * a[k];
    z[o] = s;
  }
}

typedef struct {
  double z1[HID], a1[HID], z2[HID], a2[HID], z3[HID], a3[HID], y[OUT];
} fwd_t;

static void forward(const double* w, const double* x, fwd_t* f) {
  affine(w + OFF_W1, w + OFF_B1, x, IN, HID, f->z1);
  for (int k = 0; k < HID; ++k) f->a1[k] = or_gelu(f->z1[k]);
  affine(w + OFF_W2, w + OFF_B2, f->a1, HID, HID, f->z2);
  for (int k = 0; k < HID; ++k) f->a2[k] = or_gelu(f->z2[k]);
  affine(w + OFF_W3, w + OFF_B3, f->a2, HID, HID, f->z3);
  for (int k = 0; k < HID; ++k) f->a3[k] = or_gelu(f->z3[k]);
  affine(w + OFF_W4, w + OFF_B4, f->a3, HID, OUT, f->y);
}

void or_mlp_forward(const float* params, int64_t n, const double* Xn, double* Yhat) {
  double w[NPARAM];
  load(params, w);
  for (int64_t s = 0; s < n; ++s) {
    fwd_t f;
    forward(w, Xn + s * IN, &f);
    for (int o = 0; o < OUT; ++o) Yhat[s * OUT + o] = f.y[o];
  }
}

/* Loss L = 1/(2n) sum_s sum_o (yhat - y)^2 and dL/dparams by the chain rule,
   layer by layer (backpropagation). */
void or_mlp_loss_grad(const float* params, int64_t n, const double* Xn, const double* Yn,
                      double* grad, double* loss) {
  double w[NPARAM];
  load(params, w);
  memset(grad, 0, sizeof(double) * NPARAM);
  double L = 0.0;
  for (int64_t s = 0; s < n; ++s) {
    const double* x = Xn + s * IN;
    fwd_t f;
    forward(w, x, &f);
    double d4[OUT], d3[HID], d2[HID], d1[HID];
    for (int o = 0; o < OUT; ++o) {
      const double e = f.y[o] - Yn[s * OUT + o];
      L += 0.5 * e * e / (double)n;
      d4[o] = e / (double)n;
    }
    /* output layer */
    for (int o = 0; o < OUT; ++o) {
      for (int k = 0; k < HID; ++k) grad[OFF_W4 + o * HID + k] += d4[o] * f.a3[k];
      grad[OFF_B4 + o] += d4[o];
    }
    for (int k = 0; k < HID; ++k) {
      double s3 = 0.0;
      for (int o = 0; o < OUT; ++o) s3 += w[OFF_W4 + o * HID + k] * d4[o];
      d3[k] = s3 * or_gelu_grad(f.z3[k]);
    }
    /* layer 3 */
    for (int o = 0; o < HID; ++o) {
      for (int k = 0; k < HID; ++k) grad[OFF_W3 + o * HID + k] += d3[o] * f.a2[k];
      grad[OFF_B3 + o] += d3[o];
    }
    for (int k = 0; k < HID; ++k) {
      double s2 = 0.0;
      for (int o = 0; o < HID; ++o) s2 += w[OFF_W3 + o * HID + k] * d3[o];
      d2[k] = s2 * or_gelu_grad(f.z2[k]);
    }
    /* layer 2 */
    for (int o = 0; o < HID; ++o) {
      for (int k = 0; k < HID; ++k) grad[OFF_W2 + o * HID + k] += d2[o] * f.a1[k];
      grad[OFF_B2 + o] += d2[o];
    }
    for (int k = 0; k < HID; ++k) {
      double s1 = 0.0;
      for (int o = 0; o < HID; ++o) s1 += w[OFF_W2 + o * HID + k] * d2[o];
      d1[k] = s1 * or_gelu_grad(f.z1[k]);
    }
    /* layer 1 */
    for (int o = 0; o < HID; ++o) {
      for (int k = 0; k < IN; ++k) grad[OFF_W1 + o * IN + k] += d1[o] * x[k];
      grad[OFF_B1 + o] += d1[o];
    }
  }
  *loss = L;
}

/* Adam (Kingma & Ba 2015), step number t >= 1, in FP64. */
void or_adam(int64_t n, double* p, const double* g, double* m, double* v, int64_t t, double lr,
             double b1, double b2, double eps) {
  const double c1 = 1.0 - pow(b1, (double)t), c2 = 1.0 - pow(b2, (double)t);
  for (int64_t i = 0; i < n; ++i) {
    m[i] = b1 * m[i] + (1.0 - b1) * g[i];
    v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
    p[i] -= lr * (m[i] / c1) / (sqrt(v[i] / c2) + eps);
  }
}
