/*
 * cnn_oracle.c -- plain FP64 reference of the learned warm start's network
 * (TEST INFRASTRUCTURE ONLY; the CUDA path never calls or includes it).
 *
 * Network: six 3x3x3 convolutions with zero ("same") padding and a bias,
 * channels 9 -> 24 -> 24 -> 24 -> 24 -> 24 -> 3, the Gauss-error GELU
 * g(z) = z (1 + erf(z / sqrt 2)) / 2 after layers 1-5, and a residual output
 * pred = fields + s_out * z6.  Loss: mean squared error over the in-mask
 * voxels and the 3 species.  Optimiser: Adam (Kingma & Ba 2015).
 *
 * Activity mask: the network sees the pleural space only.  A voxel is active
 * when its mask feature (input channel 8) is set; the input of layer 1 and
 * the activations a_1..a_5 are zero at inactive voxels, so an inactive voxel
 * contributes nothing to any output, as a masked (zero-flux) voxel
 * contributes nothing to the finite-volume operator of Sec. 2.4.  With every
 * voxel active this is the plain network.
 *
 * Precision model of the GPU path, reproduced here: inputs, weights and the
 * activations a_1..a_5 are rounded to bfloat16 (round to nearest even) where
 * the GPU stores them; all arithmetic is FP64 (the GPU accumulates in FP32).
 *
 * Layouts: activations [V][C] with V = nx*ny*nz, x fastest; weights of layer
 * l as [27][Ci][Co] with tap t = (dx+1) + 3((dy+1) + 3(dz+1)); biases [Co].
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

double orc_bf16(double v)
{
    float f = (float)v;
    uint32_t u;
    memcpy(&u, &f, 4);
    if ((u & 0x7f800000u) == 0x7f800000u) return (double)f;      /* inf / nan */
    const uint32_t lsb = (u >> 16) & 1u;
    u = (u + 0x7fffu + lsb) & 0xffff0000u;
    memcpy(&f, &u, 4);
    return (double)f;
}

void orc_bf16_array(int64_t n, double *a)
{
    for (int64_t i = 0; i < n; ++i) a[i] = orc_bf16(a[i]);
}

double orc_gelu(double z) { return 0.5 * z * (1.0 + erf(z / sqrt(2.0))); }

double orc_gelu_grad(double z)
{
    return 0.5 * (1.0 + erf(z / sqrt(2.0))) + z * exp(-0.5 * z * z) / sqrt(2.0 * 3.14159265358979323846);
}

/* out[v][co] = b[co] + sum_t sum_ci in[v + off(t)][ci] W[t][ci][co], zero outside. */
void orc_conv3(int nx, int ny, int nz, int Ci, int Co, const double *in, const double *W, const double *b,
               double *out)
{
    for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
        const int64_t v = i + (int64_t)nx * (j + (int64_t)ny * k);
        for (int co = 0; co < Co; ++co) out[v * Co + co] = b ? b[co] : 0.0;
        for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
            const int ii = i + dx, jj = j + dy, kk = k + dz;
            if (ii < 0 || ii >= nx || jj < 0 || jj >= ny || kk < 0 || kk >= nz) continue;
            const int t = (dx + 1) + 3 * ((dy + 1) + 3 * (dz + 1));
            const int64_t q = ii + (int64_t)nx * (jj + (int64_t)ny * kk);
            for (int ci = 0; ci < Ci; ++ci) {
                const double a = in[q * Ci + ci];
                const double *w = W + ((int64_t)t * Ci + ci) * Co;
                for (int co = 0; co < Co; ++co) out[v * Co + co] += a * w[co];
            }
        }
    }
}

/* Adjoint of orc_conv3 in its input: gin[q][ci] = sum over (v, t) with
 * q = v + off(t) of gout[v][co] W[t][ci][co]. */
void orc_conv3_dgrad(int nx, int ny, int nz, int Ci, int Co, const double *gout, const double *W, double *gin)
{
    const int64_t V = (int64_t)nx * ny * nz;
    memset(gin, 0, sizeof(double) * (size_t)(V * Ci));
    for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
        const int64_t v = i + (int64_t)nx * (j + (int64_t)ny * k);
        for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
            const int ii = i + dx, jj = j + dy, kk = k + dz;
            if (ii < 0 || ii >= nx || jj < 0 || jj >= ny || kk < 0 || kk >= nz) continue;
            const int t = (dx + 1) + 3 * ((dy + 1) + 3 * (dz + 1));
            const int64_t q = ii + (int64_t)nx * (jj + (int64_t)ny * kk);
            for (int ci = 0; ci < Ci; ++ci) {
                const double *w = W + ((int64_t)t * Ci + ci) * Co;
                double s = 0.0;
                for (int co = 0; co < Co; ++co) s += gout[v * Co + co] * w[co];
                gin[q * Ci + ci] += s;
            }
        }
    }
}

/* Gradient in the weights and bias: gW[t][ci][co] = sum_v in[v + off(t)][ci] gout[v][co]. */
void orc_conv3_wgrad(int nx, int ny, int nz, int Ci, int Co, const double *in, const double *gout, double *gW,
                     double *gb)
{
    memset(gW, 0, sizeof(double) * (size_t)(27 * Ci * Co));
    memset(gb, 0, sizeof(double) * (size_t)Co);
    for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
        const int64_t v = i + (int64_t)nx * (j + (int64_t)ny * k);
        for (int co = 0; co < Co; ++co) gb[co] += gout[v * Co + co];
        for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
            const int ii = i + dx, jj = j + dy, kk = k + dz;
            if (ii < 0 || ii >= nx || jj < 0 || jj >= ny || kk < 0 || kk >= nz) continue;
            const int t = (dx + 1) + 3 * ((dy + 1) + 3 * (dz + 1));
            const int64_t q = ii + (int64_t)nx * (jj + (int64_t)ny * kk);
            for (int ci = 0; ci < Ci; ++ci) {
                const double a = in[q * Ci + ci];
                double *g = gW + ((int64_t)t * Ci + ci) * Co;
                for (int co = 0; co < Co; ++co) g[co] += a * gout[v * Co + co];
            }
        }
    }
}

#define NL 6
static const int kCh[NL + 1] = {9, 24, 24, 24, 24, 24, 3};

/* Offsets of layer l's weights and bias in a flat parameter vector:
 * [W_1, b_1, W_2, b_2, ..., W_6, b_6]. */
int64_t orc_cnn_nparams(void)
{
    int64_t n = 0;
    for (int l = 0; l < NL; ++l) n += 27LL * kCh[l] * kCh[l + 1] + kCh[l + 1];
    return n;
}

static int64_t woff(int l)
{
    int64_t n = 0;
    for (int i = 0; i < l; ++i) n += 27LL * kCh[i] * kCh[i + 1] + kCh[i + 1];
    return n;
}

/*
 * Forward pass.  x: [V][9] input (already bf16-rounded by the caller), fields:
 * [V][3] c^n (FP64, the residual path), params: flat (bf16-rounded by the
 * caller).  z: [6][V][24] pre-activations (layer 6 uses 3 of 24 slots), a:
 * [5][V][24] activations (bf16-rounded when round_act, as on the GPU; the
 * finite-difference pins switch it off); pred: [V][3].
 */
/* The input of layer 1: x at active voxels (mask feature set), 0 elsewhere. */
static double *masked_input(int64_t V, const double *x)
{
    double *xm = (double *)malloc(sizeof(double) * (size_t)(V * 9));
    for (int64_t v = 0; v < V; ++v) {
        const int act = x[v * 9 + 8] > 0.5;
        for (int c = 0; c < 9; ++c) xm[v * 9 + c] = act ? x[v * 9 + c] : 0.0;
    }
    return xm;
}

void orc_cnn_forward(int nx, int ny, int nz, const double *x, const double *fields, const double *params,
                     double s_out, int round_act, double *z, double *a, double *pred)
{
    const int64_t V = (int64_t)nx * ny * nz;
    double *xm = masked_input(V, x);
    const double *in = xm;
    for (int l = 0; l < NL; ++l) {
        const int Ci = kCh[l], Co = kCh[l + 1];
        const double *W = params + woff(l);
        const double *b = W + 27LL * Ci * Co;
        double *zl = z + (int64_t)l * V * 24;
        orc_conv3(nx, ny, nz, Ci, Co, in, W, b, zl);
        if (l < NL - 1) {
            double *al = a + (int64_t)l * V * 24;
            for (int64_t v = 0; v < V; ++v) {
                const int act = x[v * 9 + 8] > 0.5;
                for (int c = 0; c < Co; ++c) {
                    const double g = orc_gelu(zl[v * Co + c]);
                    al[v * Co + c] = !act ? 0.0 : (round_act ? orc_bf16(g) : g);
                }
            }
            in = al;
        }
    }
    free(xm);
    const double *z6 = z + (int64_t)(NL - 1) * V * 24;
    for (int64_t v = 0; v < V; ++v)
        for (int s = 0; s < 3; ++s) pred[v * 3 + s] = fields[v * 3 + s] + s_out * z6[v * 3 + s];
}

/* Loss = sum_{v in mask, s} (pred - target)^2 / (3 * n_mask); gpred = dLoss/dpred. */
double orc_cnn_loss(int64_t V, const double *pred, const double *target, const uint8_t *mask, double *gpred)
{
    int64_t nm = 0;
    for (int64_t v = 0; v < V; ++v) nm += mask[v] ? 1 : 0;
    const double inv = nm > 0 ? 1.0 / (3.0 * (double)nm) : 0.0;
    double L = 0.0;
    for (int64_t v = 0; v < V; ++v)
        for (int s = 0; s < 3; ++s) {
            const double d = mask[v] ? pred[v * 3 + s] - target[v * 3 + s] : 0.0;
            L += d * d * inv;
            if (gpred) gpred[v * 3 + s] = 2.0 * d * inv;
        }
    return L;
}

/*
 * Backward pass from gpred = dLoss/dpred through the stored z and a (the
 * bf16 rounding of the activations is treated as the identity, a
 * straight-through derivative, as on the GPU).  The activity mask enters as
 * in the forward pass: dLoss/dz_l is zero at inactive voxels.  round_grad:
 * round each layer's dLoss/dz to bf16 where the GPU stores it (off for the
 * finite-difference pins).  Writes grads (flat, like the parameters).
 */
void orc_cnn_backward(int nx, int ny, int nz, const double *x, const double *params, double s_out,
                      const double *z, const double *a, const double *gpred, int round_grad, double *grads)
{
    const int64_t V = (int64_t)nx * ny * nz;
    double *xm = masked_input(V, x);
    double *g = (double *)malloc(sizeof(double) * (size_t)(V * 24));
    double *gp = (double *)malloc(sizeof(double) * (size_t)(V * 24));
    for (int64_t v = 0; v < V; ++v)
        for (int s = 0; s < 3; ++s) {
            const double gz = s_out * gpred[v * 3 + s];                           /* dL/dz6 */
            g[v * 3 + s] = round_grad ? orc_bf16(gz) : gz;
        }
    for (int l = NL - 1; l >= 0; --l) {
        const int Ci = kCh[l], Co = kCh[l + 1];
        const double *W = params + woff(l);
        double *gW = grads + woff(l);
        const double *in = l == 0 ? xm : a + (int64_t)(l - 1) * V * 24;
        orc_conv3_wgrad(nx, ny, nz, Ci, Co, in, g, gW, gW + 27LL * Ci * Co);
        if (l == 0) break;
        orc_conv3_dgrad(nx, ny, nz, Ci, Co, g, W, gp);                             /* dL/da_{l} */
        const double *zp = z + (int64_t)(l - 1) * V * 24;
        for (int64_t v = 0; v < V; ++v) {                                          /* dL/dz_{l} */
            const int act = x[v * 9 + 8] > 0.5;
            for (int c = 0; c < Ci; ++c) {
                const int64_t i = v * Ci + c;
                const double gz = act ? gp[i] * orc_gelu_grad(zp[i]) : 0.0;
                g[i] = round_grad ? orc_bf16(gz) : gz;
            }
        }
    }
    free(xm);
    free(g);
    free(gp);
}

/* One Adam step on n parameters (Kingma & Ba 2015, bias-corrected moments);
 * t is the 1-based step count. */
void orc_adam(int64_t n, double *p, const double *g, double *m, double *v, double lr, double b1, double b2,
              double eps, int t)
{
    const double c1 = 1.0 - pow(b1, t), c2 = 1.0 - pow(b2, t);
    for (int64_t i = 0; i < n; ++i) {
        m[i] = b1 * m[i] + (1.0 - b1) * g[i];
        v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
        p[i] -= lr * (m[i] / c1) / (sqrt(v[i] / c2) + eps);
    }
}
