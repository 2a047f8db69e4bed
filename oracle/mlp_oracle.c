/*
 * mlp_oracle.c -- plain FP64 CPU oracle of the learned warm start.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests (and nothing on the product
 * path).  Shares no code with the CUDA library.
 *
 * The network maps a normalised state to a nominal control sequence mu and a
 * per-step log sampling scale s (the warm start of Algorithm 1's U_0 and
 * Sigma_0; the paper cites learned sampling distributions as prior art, Sec. 1):
 *   h_0 = (x - x_mean) / x_std
 *   z_l = W_l h_{l-1} + b_l,  h_l = GELU(z_l) for hidden layers,
 *   y   = W_L h_{L-1} + b_L  (linear output), mu = y[0:n_mu], s = y[n_mu:n_mu+n_s]
 * with GELU(z) = z Phi(z) = z (1 + erf(z / sqrt 2)) / 2.  Loss of a batch
 * (Gaussian negative log-likelihood of the targets t, one scale per control
 * step, component j belongs to step j / nu):
 *   loss = (1/B) sum_b sum_j [ (t_j - mu_j)^2 exp(-2 s_{j/nu}) / 2 + s_{j/nu} ].
 * Adam (Kingma & Ba, 2015) with bias correction.
 *
 * Parameter layout (flat, per layer l = 1..L): W_l [d_l][d_{l-1}] row-major,
 * then b_l [d_l].
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

int64_t mlo_num_params(int32_t nlayers, const int32_t* dims) {
  int64_t p = 0;
  for (int l = 1; l <= nlayers; ++l) p += (int64_t)dims[l] * dims[l - 1] + dims[l];
  return p;
}

static double gelu(double z) { return 0.5 * z * (1.0 + erf(z / sqrt(2.0))); }
static double gelu_d(double z) {
  const double Phi = 0.5 * (1.0 + erf(z / sqrt(2.0)));
  const double phi = exp(-0.5 * z * z) / sqrt(2.0 * 3.141592653589793);
  return Phi + z * phi;
}

/* Forward pass of B samples; out: [B][d_L]. */
void mlo_forward(int32_t nlayers, const int32_t* dims, const double* params, const double* x_mean,
                 const double* x_std, int32_t B, const double* X, double* out) {
  int maxd = 0;
  for (int l = 0; l <= nlayers; ++l)
    if (dims[l] > maxd) maxd = dims[l];
  double* h = (double*)malloc(sizeof(double) * maxd);
  double* z = (double*)malloc(sizeof(double) * maxd);
  for (int b = 0; b < B; ++b) {
    for (int i = 0; i < dims[0]; ++i) h[i] = (X[(int64_t)b * dims[0] + i] - x_mean[i]) / x_std[i];
    const double* p = params;
    for (int l = 1; l <= nlayers; ++l) {
      const int din = dims[l - 1], dout = dims[l];
      const double* W = p;
      const double* bias = p + (int64_t)dout * din;
      for (int o = 0; o < dout; ++o) {
        double acc = bias[o];
        for (int i = 0; i < din; ++i) acc += W[(int64_t)o * din + i] * h[i];
        z[o] = acc;
      }
      for (int o = 0; o < dout; ++o) h[o] = (l < nlayers) ? gelu(z[o]) : z[o];
      p += (int64_t)dout * din + dout;
    }
    memcpy(out + (int64_t)b * dims[nlayers], h, sizeof(double) * dims[nlayers]);
  }
  free(h);
  free(z);
}

/* Loss and gradient (grad: same layout as params) of one batch.  T: [B][n_mu]
 * targets; the output layer has n_mu + n_mu / nu units. */
double mlo_loss_grad(int32_t nlayers, const int32_t* dims, const double* params, const double* x_mean,
                     const double* x_std, int32_t B, const double* X, const double* T, int32_t nu, double* grad) {
  const int64_t np = mlo_num_params(nlayers, dims);
  const int nmu = dims[nlayers] * nu / (nu + 1);
  int maxd = 0;
  for (int l = 0; l <= nlayers; ++l)
    if (dims[l] > maxd) maxd = dims[l];
  /* activations per layer: h[l] (post-activation), z[l] (pre-activation) */
  double** hs = (double**)malloc(sizeof(double*) * (nlayers + 1));
  double** zs = (double**)malloc(sizeof(double*) * (nlayers + 1));
  for (int l = 0; l <= nlayers; ++l) {
    hs[l] = (double*)malloc(sizeof(double) * dims[l]);
    zs[l] = (double*)malloc(sizeof(double) * dims[l]);
  }
  double* dh = (double*)malloc(sizeof(double) * maxd);
  double* dz = (double*)malloc(sizeof(double) * maxd);
  memset(grad, 0, sizeof(double) * (size_t)np);
  double loss = 0.0;
  for (int b = 0; b < B; ++b) {
    for (int i = 0; i < dims[0]; ++i) hs[0][i] = (X[(int64_t)b * dims[0] + i] - x_mean[i]) / x_std[i];
    const double* p = params;
    for (int l = 1; l <= nlayers; ++l) {
      const int din = dims[l - 1], dout = dims[l];
      const double* W = p;
      const double* bias = p + (int64_t)dout * din;
      for (int o = 0; o < dout; ++o) {
        double acc = bias[o];
        for (int i = 0; i < din; ++i) acc += W[(int64_t)o * din + i] * hs[l - 1][i];
        zs[l][o] = acc;
        hs[l][o] = (l < nlayers) ? gelu(acc) : acc;
      }
      p += (int64_t)dout * din + dout;
    }
    /* loss of this sample and dL/dy */
    const double* y = hs[nlayers];
    const double* t = T + (int64_t)b * nmu;
    for (int o = 0; o < dims[nlayers]; ++o) dz[o] = 0.0;
    for (int j = 0; j < nmu; ++j) {
      const int k = j / nu;
      const double sk = y[nmu + k];
      const double e = t[j] - y[j];
      const double w = exp(-2.0 * sk);
      loss += 0.5 * e * e * w + sk;
      dz[j] += -e * w / B;
      dz[nmu + k] += (-e * e * w + 1.0) / B;
    }
    /* backward through the layers */
    int64_t off = np;
    for (int l = nlayers; l >= 1; --l) {
      const int din = dims[l - 1], dout = dims[l];
      off -= (int64_t)dout * din + dout;
      const double* W = params + off;
      double* gW = grad + off;
      double* gb = gW + (int64_t)dout * din;
      for (int o = 0; o < dout; ++o) {
        gb[o] += dz[o];
        for (int i = 0; i < din; ++i) gW[(int64_t)o * din + i] += dz[o] * hs[l - 1][i];
      }
      if (l > 1) {
        for (int i = 0; i < din; ++i) {
          double acc = 0.0;
          for (int o = 0; o < dout; ++o) acc += W[(int64_t)o * din + i] * dz[o];
          dh[i] = acc;
        }
        for (int i = 0; i < din; ++i) dz[i] = dh[i] * gelu_d(zs[l - 1][i]);
      }
    }
  }
  for (int l = 0; l <= nlayers; ++l) {
    free(hs[l]);
    free(zs[l]);
  }
  free(hs);
  free(zs);
  free(dh);
  free(dz);
  return loss / B;
}

/* One Adam step (step index t >= 1) on every parameter. */
void mlo_adam(int64_t np, double* params, const double* grad, double* m, double* v, int32_t t, double lr, double b1,
              double b2, double eps) {
  const double c1 = 1.0 - pow(b1, t), c2 = 1.0 - pow(b2, t);
  for (int64_t i = 0; i < np; ++i) {
    m[i] = b1 * m[i] + (1.0 - b1) * grad[i];
    v[i] = b2 * v[i] + (1.0 - b2) * grad[i] * grad[i];
    const double mh = m[i] / c1, vh = v[i] / c2;
    params[i] -= lr * mh / (sqrt(vh) + eps);
  }
}
