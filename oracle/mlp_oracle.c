/*
 * FP64 CPU oracle of the surrogate network that warm-starts the game
 * iteration: a multilayer perceptron in -> hidden (x L) -> out with GELU
 * activations between layers and a linear output, and its mean-squared-error
 * gradient by backpropagation, plus one Adam step.
 *
 * TEST INFRASTRUCTURE ONLY (gradient checks of the GPU kernels); the paper
 * initialises the iteration with "some given" values (Section 2.1, Step 0) and
 * has no network. The definitions used:
 *   GELU(z) = z Phi(z) = z (1 + erf(z / sqrt 2)) / 2,
 *   GELU'(z) = Phi(z) + z phi(z),  phi(z) = exp(-z^2/2) / sqrt(2 pi),
 *   loss = (1 / (B * out)) sum_{b,o} (y_{b,o} - t_{b,o})^2,
 *   Adam (Kingma & Ba 2015): m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
 *   w -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
 * Parameter layout (flat): for each layer l, W_l (n_out x n_in, row-major)
 * followed by b_l (n_out).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

double orc_gelu(double z) { return 0.5 * z * (1.0 + erf(z / sqrt(2.0))); }

double orc_gelu_grad(double z)
{
    const double Phi = 0.5 * (1.0 + erf(z / sqrt(2.0)));
    const double phi = exp(-0.5 * z * z) / sqrt(2.0 * 3.14159265358979323846);
    return Phi + z * phi;
}

/* dims[0..L]: layer widths (dims[0] = inputs, dims[L] = outputs), L layers.
 * Z (optional): pre-activations of every layer, sum_l B dims[l+1] doubles;
 * H (optional): activations, the same size (the last layer's H = Z). */
static void forward_all(int L, const int *dims, const double *params, int B, const double *X, double *Z,
                        double *H)
{
    const double *p = params;
    const double *in = X;
    size_t off = 0;
    for (int l = 0; l < L; ++l) {
        const int ni = dims[l], no = dims[l + 1];
        const double *W = p, *bias = p + (size_t)no * ni;
        for (int b = 0; b < B; ++b)
            for (int o = 0; o < no; ++o) {
                double s = bias[o];
                for (int k = 0; k < ni; ++k) s += W[(size_t)o * ni + k] * in[(size_t)b * ni + k];
                Z[off + (size_t)b * no + o] = s;
                H[off + (size_t)b * no + o] = (l < L - 1) ? orc_gelu(s) : s;
            }
        in = H + off;
        off += (size_t)B * no;
        p += (size_t)no * ni + no;
    }
}

static size_t act_size(int L, const int *dims, int B)
{
    size_t s = 0;
    for (int l = 0; l < L; ++l) s += (size_t)B * dims[l + 1];
    return s;
}

void orc_mlp_forward(int L, const int *dims, const double *params, int B, const double *X, double *Y,
                     double *unused)
{
    (void)unused;
    size_t n = act_size(L, dims, B);
    double *Z = (double *)malloc(sizeof(double) * n);
    double *H = (double *)malloc(sizeof(double) * n);
    forward_all(L, dims, params, B, X, Z, H);
    memcpy(Y, H + n - (size_t)B * dims[L], sizeof(double) * (size_t)B * dims[L]);
    free(Z);
    free(H);
}

/* Loss and its gradient with respect to every parameter (same flat layout). */
double orc_mlp_loss_grad(int L, const int *dims, const double *params, int B, const double *X,
                         const double *T, double *grad, double *unused)
{
    (void)unused;
    size_t n = act_size(L, dims, B);
    double *Z = (double *)malloc(sizeof(double) * n);
    double *H = (double *)malloc(sizeof(double) * n);
    forward_all(L, dims, params, B, X, Z, H);
    const int nout = dims[L];
    const size_t yoff = n - (size_t)B * nout;
    double loss = 0.0;
    int maxw = 0;
    for (int l = 0; l <= L; ++l) if (dims[l] > maxw) maxw = dims[l];
    double *dZ = (double *)malloc(sizeof(double) * (size_t)B * maxw);
    double *dH = (double *)malloc(sizeof(double) * (size_t)B * maxw);
    const double scale = 1.0 / ((double)B * nout);
    for (int b = 0; b < B; ++b)
        for (int o = 0; o < nout; ++o) {
            const double d = H[yoff + (size_t)b * nout + o] - T[(size_t)b * nout + o];
            loss += d * d * scale;
            dZ[(size_t)b * nout + o] = 2.0 * d * scale;
        }
    /* parameter offsets */
    size_t *poff = (size_t *)malloc(sizeof(size_t) * (size_t)(L + 1));
    poff[0] = 0;
    for (int l = 0; l < L; ++l) poff[l + 1] = poff[l] + (size_t)dims[l + 1] * dims[l] + dims[l + 1];
    size_t aoff = yoff;   /* offset of layer l's activations */
    for (int l = L - 1; l >= 0; --l) {
        const int ni = dims[l], no = dims[l + 1];
        const double *W = params + poff[l];
        double *gW = grad + poff[l], *gb = gW + (size_t)no * ni;
        const double *in = (l == 0) ? X : H + (aoff - (size_t)B * ni);
        for (int o = 0; o < no; ++o) {
            double sb = 0.0;
            for (int b = 0; b < B; ++b) sb += dZ[(size_t)b * no + o];
            gb[o] = sb;
            for (int k = 0; k < ni; ++k) {
                double s = 0.0;
                for (int b = 0; b < B; ++b) s += dZ[(size_t)b * no + o] * in[(size_t)b * ni + k];
                gW[(size_t)o * ni + k] = s;
            }
        }
        if (l > 0) {
            const size_t zoff = aoff - (size_t)B * ni;   /* pre-activations of layer l-1 */
            for (int b = 0; b < B; ++b)
                for (int k = 0; k < ni; ++k) {
                    double s = 0.0;
                    for (int o = 0; o < no; ++o) s += dZ[(size_t)b * no + o] * W[(size_t)o * ni + k];
                    dH[(size_t)b * ni + k] = s * orc_gelu_grad(Z[zoff + (size_t)b * ni + k]);
                }
            memcpy(dZ, dH, sizeof(double) * (size_t)B * ni);
            aoff = zoff;
        }
    }
    free(poff);
    free(dZ);
    free(dH);
    free(Z);
    free(H);
    return loss;
}

/* One Adam step (t = step count after this update, starting at 1). */
void orc_adam_step(long n, double *w, const double *g, double *m, double *v, double lr, double b1, double b2,
                   double eps, long t)
{
    const double c1 = 1.0 - pow(b1, (double)t), c2 = 1.0 - pow(b2, (double)t);
    for (long i = 0; i < n; ++i) {
        m[i] = b1 * m[i] + (1.0 - b1) * g[i];
        v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
        w[i] -= lr * (m[i] / c1) / (sqrt(v[i] / c2) + eps);
    }
}
