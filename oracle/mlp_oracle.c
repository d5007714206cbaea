/*
 * mlp_oracle.c -- FP64 oracle of the learned screen's network (TEST
 * INFRASTRUCTURE ONLY; shares no code with the CUDA library).
 *
 * Network: 12 features -> 64 (ReLU) -> 64 (ReLU) -> 1 (sigmoid), trained with
 * the mean binary cross-entropy.  The library computes with BF16 operands and
 * FP32 accumulation; this oracle computes in FP64 but rounds every operand the
 * library feeds to a BF16 product to BF16 at the same place: the inputs, the
 * weights, the hidden activations entering layers 2 and 3, and the
 * back-propagated activation gradients entering the BF16 products of the
 * backward pass.  BF16 rounding is round-to-nearest-even on the float32 value
 * (IEEE 754 binary16-brain: keep the top 16 bits of binary32).
 *
 * Parameter layout (5,057 floats): W1[12][64] (row = input), b1[64],
 * W2[64][64] (row = input), b2[64], W3[64], b3.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#define NF 12
#define NH 64
#define OFF_W1 0
#define OFF_B1 (NF * NH)
#define OFF_W2 (OFF_B1 + NH)
#define OFF_B2 (OFF_W2 + NH * NH)
#define OFF_W3 (OFF_B2 + NH)
#define OFF_B3 (OFF_W3 + NH)
#define NPARAM (OFF_B3 + 1)

int orc_mlp_nparams(void) { return NPARAM; }

/* Round a float to the nearest BF16 value (ties to even), returned as float. */
float orc_bf16(float x) {
  uint32_t u;
  memcpy(&u, &x, 4);
  if ((u & 0x7f800000u) == 0x7f800000u) { /* inf / nan: truncate */
    u &= 0xffff0000u;
  } else {
    uint32_t lsb = (u >> 16) & 1u;
    u += 0x7fffu + lsb;
    u &= 0xffff0000u;
  }
  float y;
  memcpy(&y, &u, 4);
  return y;
}

static double b16(double x) { return (double)orc_bf16((float)x); }

/* Forward pass for n rows of X (n x 12, float32).  p_out (may be NULL)
 * receives the probabilities; returns the mean BCE against y (if y != NULL). */
double orc_mlp_forward(const float* P, const float* X, const float* y, int64_t n, double* p_out) {
  double loss = 0.0;
  for (int64_t r = 0; r < n; r++) {
    double x[NF], h1[NH], h2[NH];
    for (int i = 0; i < NF; i++) x[i] = b16(X[r * NF + i]);
    for (int j = 0; j < NH; j++) {
      double s = 0;
      for (int i = 0; i < NF; i++) s += x[i] * b16(P[OFF_W1 + i * NH + j]);
      s += P[OFF_B1 + j];
      h1[j] = b16(s > 0 ? s : 0);
    }
    for (int j = 0; j < NH; j++) {
      double s = 0;
      for (int i = 0; i < NH; i++) s += h1[i] * b16(P[OFF_W2 + i * NH + j]);
      s += P[OFF_B2 + j];
      h2[j] = b16(s > 0 ? s : 0);
    }
    double z = P[OFF_B3];
    for (int i = 0; i < NH; i++) z += h2[i] * b16(P[OFF_W3 + i]);
    double p = 1.0 / (1.0 + exp(-z));
    if (p_out) p_out[r] = p;
    if (y) {
      /* BCE from the logit, stable form: max(z,0) - z y + log(1 + e^-|z|) */
      double t = y[r];
      loss += (z > 0 ? z : 0) - z * t + log1p(exp(-fabs(z)));
    }
  }
  return n ? loss / (double)n : 0.0;
}

/* Mean BCE and its gradient with respect to all 5,057 parameters. */
double orc_mlp_grad(const float* P, const float* X, const float* y, int64_t n, double* G) {
  for (int k = 0; k < NPARAM; k++) G[k] = 0;
  double loss = 0;
  for (int64_t r = 0; r < n; r++) {
    double x[NF], z1[NH], h1[NH], z2[NH], h2[NH];
    for (int i = 0; i < NF; i++) x[i] = b16(X[r * NF + i]);
    for (int j = 0; j < NH; j++) {
      double s = 0;
      for (int i = 0; i < NF; i++) s += x[i] * b16(P[OFF_W1 + i * NH + j]);
      z1[j] = s + P[OFF_B1 + j];
      h1[j] = b16(z1[j] > 0 ? z1[j] : 0);
    }
    for (int j = 0; j < NH; j++) {
      double s = 0;
      for (int i = 0; i < NH; i++) s += h1[i] * b16(P[OFF_W2 + i * NH + j]);
      z2[j] = s + P[OFF_B2 + j];
      h2[j] = b16(z2[j] > 0 ? z2[j] : 0);
    }
    double z = P[OFF_B3];
    for (int i = 0; i < NH; i++) z += h2[i] * b16(P[OFF_W3 + i]);
    const double p = 1.0 / (1.0 + exp(-z));
    const double t = y[r];
    loss += (z > 0 ? z : 0) - z * t + log1p(exp(-fabs(z)));
    const double dz = (p - t) / (double)n;  /* d(mean BCE)/dz */
    /* layer 3 */
    double dh2[NH];
    for (int i = 0; i < NH; i++) {
      G[OFF_W3 + i] += h2[i] * dz;
      dh2[i] = z2[i] > 0 ? b16(dz * b16(P[OFF_W3 + i])) : 0;
    }
    G[OFF_B3] += dz;
    /* layer 2 */
    double dh1[NH];
    for (int i = 0; i < NH; i++) {
      double s = 0;
      for (int j = 0; j < NH; j++) s += dh2[j] * b16(P[OFF_W2 + i * NH + j]);
      dh1[i] = z1[i] > 0 ? b16(s) : 0;
    }
    for (int i = 0; i < NH; i++)
      for (int j = 0; j < NH; j++) G[OFF_W2 + i * NH + j] += h1[i] * dh2[j];
    for (int j = 0; j < NH; j++) G[OFF_B2 + j] += dh2[j];
    /* layer 1 */
    for (int i = 0; i < NF; i++)
      for (int j = 0; j < NH; j++) G[OFF_W1 + i * NH + j] += x[i] * dh1[j];
    for (int j = 0; j < NH; j++) G[OFF_B1 + j] += dh1[j];
  }
  return n ? loss / (double)n : 0.0;
}

/* The same loss and gradient with no BF16 rounding anywhere (pure FP64):
 * the reference for finite-difference checks. */
double orc_mlp_grad_exact(const double* P, const double* X, const double* y, int64_t n, double* G) {
  for (int k = 0; k < NPARAM; k++) G[k] = 0;
  double loss = 0;
  for (int64_t r = 0; r < n; r++) {
    double z1[NH], h1[NH], z2[NH], h2[NH];
    const double* x = X + r * NF;
    for (int j = 0; j < NH; j++) {
      double s = P[OFF_B1 + j];
      for (int i = 0; i < NF; i++) s += x[i] * P[OFF_W1 + i * NH + j];
      z1[j] = s;
      h1[j] = s > 0 ? s : 0;
    }
    for (int j = 0; j < NH; j++) {
      double s = P[OFF_B2 + j];
      for (int i = 0; i < NH; i++) s += h1[i] * P[OFF_W2 + i * NH + j];
      z2[j] = s;
      h2[j] = s > 0 ? s : 0;
    }
    double z = P[OFF_B3];
    for (int i = 0; i < NH; i++) z += h2[i] * P[OFF_W3 + i];
    const double p = 1.0 / (1.0 + exp(-z));
    const double t = y[r];
    loss += (z > 0 ? z : 0) - z * t + log1p(exp(-fabs(z)));
    const double dz = (p - t) / (double)n;
    double dh2[NH], dh1[NH];
    for (int i = 0; i < NH; i++) {
      G[OFF_W3 + i] += h2[i] * dz;
      dh2[i] = z2[i] > 0 ? dz * P[OFF_W3 + i] : 0;
    }
    G[OFF_B3] += dz;
    for (int i = 0; i < NH; i++) {
      double s = 0;
      for (int j = 0; j < NH; j++) s += dh2[j] * P[OFF_W2 + i * NH + j];
      dh1[i] = z1[i] > 0 ? s : 0;
    }
    for (int i = 0; i < NH; i++)
      for (int j = 0; j < NH; j++) G[OFF_W2 + i * NH + j] += h1[i] * dh2[j];
    for (int j = 0; j < NH; j++) G[OFF_B2 + j] += dh2[j];
    for (int i = 0; i < NF; i++)
      for (int j = 0; j < NH; j++) G[OFF_W1 + i * NH + j] += x[i] * dh1[j];
    for (int j = 0; j < NH; j++) G[OFF_B1 + j] += dh1[j];
  }
  return n ? loss / (double)n : 0.0;
}

double orc_mlp_loss_exact(const double* P, const double* X, const double* y, int64_t n) {
  double G[NPARAM];
  return orc_mlp_grad_exact(P, X, y, n, G);
}
