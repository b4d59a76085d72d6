/*
 * mlp_oracle.c -- FP64 reference of the interceptor-ranking network (TEST
 * INFRASTRUCTURE: only the tests, the smoke check and the bench's CPU leg load it).
 *
 * The network scores a candidate interceptor z of a candidate pair (x, y) from 32
 * features: two hidden layers of 128 rectified linear units and one output logit,
 *     h1 = relu(W1 f + b1),  h2 = relu(W2 h1 + b2),  s = w3 . h2 + b3.
 * It extends the paper's Stage V (the "select group" of likely interceptors tried
 * before the exhaustive Stage VI search): a pair tries the k best-scored candidates
 * first, and the exact test of Eq. 1 decides as before.
 *
 * Parameter vector (doubles, in this order): W1[128][32] (row = hidden unit),
 * b1[128], W2[128][128] (row = unit of the second layer), b2[128], w3[128], b3.
 *
 * Loss of a batch: L = (1/N) sum_b w_b [ log(1 + exp(s_b)) - y_b s_b ]
 * (logistic loss on the logit, weight w_b per sample).  The gradient is written
 * out by the chain rule, layer by layer, with relu'(0) = 0.
 *
 * Plain loops in the order of the formulas; no blocking and no reordering.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define MLP_IN 32
#define MLP_H 128
#define OFF_W1 0
#define OFF_B1 (OFF_W1 + MLP_H * MLP_IN)
#define OFF_W2 (OFF_B1 + MLP_H)
#define OFF_B2 (OFF_W2 + MLP_H * MLP_H)
#define OFF_W3 (OFF_B2 + MLP_H)
#define OFF_B3 (OFF_W3 + MLP_H)
#define MLP_NPARAM (OFF_B3 + 1)

int64_t orc_mlp_nparams(void) { return MLP_NPARAM; }

/* forward pass of one sample; z1, h1, z2, h2 receive the layer values */
static double forward1(const double* P, const double* f, double* z1, double* h1, double* z2, double* h2) {
  for (int j = 0; j < MLP_H; ++j) {
    double a = P[OFF_B1 + j];
    for (int k = 0; k < MLP_IN; ++k) a += P[OFF_W1 + j * MLP_IN + k] * f[k];
    z1[j] = a;
    h1[j] = a > 0.0 ? a : 0.0;
  }
  for (int j = 0; j < MLP_H; ++j) {
    double a = P[OFF_B2 + j];
    for (int i = 0; i < MLP_H; ++i) a += P[OFF_W2 + j * MLP_H + i] * h1[i];
    z2[j] = a;
    h2[j] = a > 0.0 ? a : 0.0;
  }
  double s = P[OFF_B3];
  for (int j = 0; j < MLP_H; ++j) s += P[OFF_W3 + j] * h2[j];
  return s;
}

/* logits[b] for the N samples X[N][32] */
void orc_mlp_forward(const double* P, const double* X, int64_t N, double* logits) {
  double z1[MLP_H], h1[MLP_H], z2[MLP_H], h2[MLP_H];
  for (int64_t b = 0; b < N; ++b) logits[b] = forward1(P, X + b * MLP_IN, z1, h1, z2, h2);
}

/* log(1 + exp(s)) without overflow */
static double softplus(double s) { return s > 0.0 ? s + log1p(exp(-s)) : log1p(exp(s)); }

/* loss of the batch; grad[MLP_NPARAM] receives dL/dP (overwritten) */
double orc_mlp_backward(const double* P, const double* X, const double* y, const double* w, int64_t N,
                        double* grad) {
  double z1[MLP_H], h1[MLP_H], z2[MLP_H], h2[MLP_H], d2[MLP_H], d1[MLP_H];
  memset(grad, 0, sizeof(double) * MLP_NPARAM);
  double loss = 0.0;
  for (int64_t b = 0; b < N; ++b) {
    const double* f = X + b * MLP_IN;
    const double s = forward1(P, f, z1, h1, z2, h2);
    const double wb = w ? w[b] : 1.0;
    loss += wb * (softplus(s) - y[b] * s);
    /* dL/ds = w (sigmoid(s) - y) / N */
    const double ds = wb * (1.0 / (1.0 + exp(-s)) - y[b]) / (double)N;
    grad[OFF_B3] += ds;
    for (int j = 0; j < MLP_H; ++j) {
      grad[OFF_W3 + j] += ds * h2[j];
      d2[j] = z2[j] > 0.0 ? ds * P[OFF_W3 + j] : 0.0; /* dL/dz2 */
    }
    for (int j = 0; j < MLP_H; ++j) {
      grad[OFF_B2 + j] += d2[j];
      for (int i = 0; i < MLP_H; ++i) grad[OFF_W2 + j * MLP_H + i] += d2[j] * h1[i];
    }
    for (int i = 0; i < MLP_H; ++i) {
      double a = 0.0;
      for (int j = 0; j < MLP_H; ++j) a += P[OFF_W2 + j * MLP_H + i] * d2[j];
      d1[i] = z1[i] > 0.0 ? a : 0.0; /* dL/dz1 */
    }
    for (int j = 0; j < MLP_H; ++j) {
      grad[OFF_B1 + j] += d1[j];
      for (int k = 0; k < MLP_IN; ++k) grad[OFF_W1 + j * MLP_IN + k] += d1[j] * f[k];
    }
  }
  return loss / (double)N;
}
