/*
 * lsd_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded FP64 reference of Langevin Speculative
 * Dynamics (LSD, "Speculative Sampling For Faster Molecular Dynamics").  It
 * exists so that tests and the benchmark's CPU baseline can check the CUDA
 * library against something that can be read against the paper by eye.  It
 * shares no code, header, table or constant generator with the CUDA library,
 * and nothing in the product path may link or call it.
 *
 * Everything is FP64 except the neighbour membership rule, which is a discrete
 * definition (the paper uses external force fields and is silent on it) and is
 * written out in o_member() below.
 *
 * Units: positions in Angstrom, time in fs, mass in amu, energy in eV,
 * momentum in amu*Angstrom/fs.  KAPPA converts a force in eV/Angstrom into
 * amu*Angstrom/fs^2.
 *
 * Parity pins (tests/test_oracle_*.py): Philox known-answer vectors, finite
 * differences of the energy (forces), two-/three-atom closed forms
 * (LJ, radial, angular), a periodic lattice sum (image handling), the 1-D
 * reflection coupling, the erf rejection law (Eq. 6), a KS test of transported
 * momenta (Eq. 3 / Thm 3.1), the harmonic ABOBA stationary covariance
 * (discrete Lyapunov equation), draft == target giving plain ABOBA bit for bit,
 * and window-length invariance of the committed trajectory (Alg. 1).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define O_PI 3.14159265358979323846
#define O_TWO32 4294967296.0

/* CODATA 2018: 1 eV = 1.602176634e-19 J, 1 amu = 1.66053906660e-27 kg,
 * k_B = 1.380649e-23 J/K. */
static double o_kappa(void) {
    /* (1 eV/Angstrom in N) / (1 amu*Angstrom/fs^2 in N) */
    return (1.602176634e-19 / 1e-10) / (1.66053906660e-27 * 1e-10 / 1e-30);
}
static double o_kboltz(void) { return 1.380649e-23 / 1.602176634e-19; } /* eV/K */

double o_const_kappa(void) { return o_kappa(); }
double o_const_kb(void) { return o_kboltz(); }

/* ------------------------------------------------------------------------- */
/* Interfaces                                                                 */
/* ------------------------------------------------------------------------- */

typedef struct {
    int32_t n_atoms;
    int32_t n_species;
    double box[3];               /* orthorhombic periodic box, Angstrom */
    const int32_t *species;      /* [N] */
    const double *species_mass;  /* [n_species], amu */
} o_system;

enum { O_HEAD_TANH = 0, O_HEAD_LINEAR = 1 };

typedef struct {
    /* Lennard-Jones term, active when lj_cutoff > 0 */
    const double *lj_eps;        /* [n_species], eV */
    const double *lj_sigma;      /* [n_species], Angstrom */
    double lj_cutoff;
    /* per-atom MLP on descriptors, active when n_layers > 0 */
    int32_t n_rbf, n_ang, n_layers, width;
    double desc_cutoff;
    int32_t head;                /* O_HEAD_TANH: head_scale*tanh(y); O_HEAD_LINEAR: y */
    double head_scale;
    const double *weights;       /* packed, see o_n_weights() */
    /* harmonic tether 0.5*k*|q - q_ref|^2 (no periodic images), active when k_harm > 0 */
    double k_harm;
    const double *q_ref;         /* [3N] */
    /* non-conservative shear field F_x += shear*sin(2*pi*y/L_y), active when != 0 */
    double shear;
} o_potential;

enum { O_ABOBA = 0, O_OBABO = 1 };

typedef struct {
    double dt;          /* fs */
    double gamma;       /* 1/fs */
    double temperature; /* K */
    uint64_t seed;
    int32_t integrator; /* O_ABOBA (Eq. 2), or O_OBABO in the staggered frame of App. E */
} o_params;

int32_t o_input_dim(int32_t n_species, int32_t n_rbf, int32_t n_ang) {
    return n_species * n_rbf + n_ang + n_species;
}

/* Packed MLP parameters: for each hidden layer l: W_l [width][d_in] row-major,
 * then b_l [width]; then the output row w_out [width] and b_out [1]. */
int64_t o_n_weights(int32_t d0, int32_t n_layers, int32_t width) {
    if (n_layers <= 0) return 0;
    int64_t n = (int64_t)width * d0 + width;
    n += (int64_t)(n_layers - 1) * ((int64_t)width * width + width);
    n += width + 1;
    return n;
}

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), written from its        */
/* published definition: 10 rounds of the 4x32 multiply-xor bijection with a  */
/* Weyl-sequence key schedule.                                                */
/* ------------------------------------------------------------------------- */

void o_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void o_philox_words(uint64_t seed, uint64_t n, uint32_t atom, uint32_t stream, uint32_t w[4]) {
    uint32_t ctr[4] = {(uint32_t)n, (uint32_t)(n >> 32), atom, stream};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    o_philox4x32_10(ctr, key, w);
}

/* Three standard normals for (step n, atom, stream) by the Box-Muller transform
 * on 23-bit uniforms: u1 = ((w0>>9)+1/2)/2^23 in (0,1), u2 = (w1>>9)/2^23 in
 * [0,1); x = sqrt(-2 ln u1) cos(2 pi u2), y = ... sin(...); z from (w2, w3),
 * its sine partner dropped. */
void o_normals(uint64_t seed, uint64_t n, uint32_t atom, uint32_t stream, double xi[3]) {
    uint32_t w[4];
    o_philox_words(seed, n, atom, stream, w);
    double u1 = ((double)(w[0] >> 9) + 0.5) * 0x1p-23;
    double u2 = (double)(w[1] >> 9) * 0x1p-23;
    double u3 = ((double)(w[2] >> 9) + 0.5) * 0x1p-23;
    double u4 = (double)(w[3] >> 9) * 0x1p-23;
    double r1 = sqrt(-2.0 * log(u1));
    double r2 = sqrt(-2.0 * log(u3));
    xi[0] = r1 * cos(2.0 * O_PI * u2);
    xi[1] = r1 * sin(2.0 * O_PI * u2);
    xi[2] = r2 * cos(2.0 * O_PI * u4);
}

/* Uniform in (0, 1] with 53 random bits for the acceptance test of step n:
 * ((w0>>5)*2^26 + (w1>>6) + 1) / 2^53, stream 1, atom field 0. */
double o_uniform(uint64_t seed, uint64_t n) {
    uint32_t w[4];
    o_philox_words(seed, n, 0u, 1u, w);
    uint64_t m = (uint64_t)(w[0] >> 5) * 67108864ull + (uint64_t)(w[1] >> 6) + 1ull;
    return (double)m * 0x1p-53;
}

/* ------------------------------------------------------------------------- */
/* Neighbour membership rule                                                  */
/* ------------------------------------------------------------------------- */
/* Each coordinate is mapped to 32-bit fixed point: t = q * (2^32 / L),
 * f = floor(t), u = f mod 2^32 (the wrapped position in units of L/2^32) and
 * m = (f - u) / 2^32 (the periodic image count).  Along one axis the pair
 * (i, j) has the wrapped difference d0 = (int32)(u_j - u_i mod 2^32) (the
 * minimum image in fixed point, k = (u_j - u_i - d0)/2^32 in {-1,0,1} images
 * away from the unwrapped difference), the minimum-image displacement
 * dmin = fl32(fl32(d0) * fl32(L/2^32)), and for the image r in {-1,0,1}
 * relative to it the displacement d_r = dmin (r = 0) or fl32(dmin + r*fl32(L)).
 * The absolute image shift of that displacement is s = r - k.  A pair (i, j, s)
 * is a member iff every axis has |r| <= 1 and ((dx*dx + dy*dy) + dz*dz) <
 * fl32(rc^2) in binary32 without fused multiply-add.  Self pairs are excluded
 * only for s = 0.  The shift code is (sx+1) + 3(sy+1) + 9(sz+1).  Requires
 * rc < L on every axis (then no image with |r| > 1 can be within reach). */

typedef struct { uint32_t u[3]; int64_t m[3]; } o_fix;

static void o_fixpoint(const o_system *sys, const double *q, o_fix *fx) {
    for (int i = 0; i < sys->n_atoms; ++i) {
        for (int a = 0; a < 3; ++a) {
            double scale = O_TWO32 / sys->box[a];
            double t = q[3 * i + a] * scale;
            double f = floor(t);
            int64_t fi = (int64_t)f;
            uint32_t u = (uint32_t)((uint64_t)fi & 0xFFFFFFFFull);
            fx[i].u[a] = u;
            fx[i].m[a] = (fi - (int64_t)u) / (int64_t)4294967296ll;
        }
    }
}

static int o_member(const o_system *sys, const o_fix *fx, int i, int j, const int s[3], float rc2f,
                    float *d2_out) {
    float d[3];
    for (int a = 0; a < 3; ++a) {
        uint32_t ui = fx[i].u[a], uj = fx[j].u[a];
        int32_t d0 = (int32_t)(uint32_t)(uj - ui);
        int64_t D0 = (int64_t)uj - (int64_t)ui;
        int k = (int)((D0 - (int64_t)d0) / 4294967296ll);
        int r = s[a] + k;
        if (r < -1 || r > 1) return 0;
        float scale_f = (float)(sys->box[a] / O_TWO32);
        float Lf = (float)sys->box[a];
        float dmin = (float)d0 * scale_f;
        d[a] = (r == 0) ? dmin : dmin + (float)r * Lf;
    }
    float xx = d[0] * d[0];
    float yy = d[1] * d[1];
    float zz = d[2] * d[2];
    float d2 = xx + yy;
    d2 = d2 + zz;
    if (d2_out) *d2_out = d2;
    return d2 < rc2f;
}

/* FP64 displacement from atom i to the image s of atom j, consistent with the
 * fixed-point wrap above. */
static void o_disp(const o_system *sys, const double *q, const o_fix *fx, int i, int j, const int s[3],
                   double d[3]) {
    for (int a = 0; a < 3; ++a) {
        double shift = (double)((int64_t)s[a] - fx[j].m[a] + fx[i].m[a]);
        d[a] = (q[3 * j + a] - q[3 * i + a]) + shift * sys->box[a];
    }
}

typedef struct { int32_t j; int32_t code; double d[3]; double r; } o_nb;

/* Brute-force neighbour list of atom i within rc, in canonical order
 * (neighbour index ascending, then shift code ascending). */
/* A conservative pre-test that changes no list: along every axis each image
 * other than the minimum one is at least as far as it (|d0| <= 2^31, so the
 * minimum-image displacement is at most L/2), so when the minimum-image
 * distance, in FP64 from the same fixed-point coordinates, exceeds the cutoff
 * by more than the rule's FP32 rounding could hide (1e-5 relative, against a
 * few 1e-7), no image of j passes the rule.  o_set_list_prefilter(0) turns it
 * off (the tests compare both). */
static int o_prefilter = 1;

void o_set_list_prefilter(int32_t on) { o_prefilter = on != 0; }

static int o_beyond(const o_system *sys, const o_fix *fx, int i, int j, double rc2) {
    double d2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        int32_t d0 = (int32_t)(uint32_t)(fx[j].u[a] - fx[i].u[a]);
        double d = (double)d0 * (sys->box[a] / O_TWO32);
        d2 += d * d;
    }
    return d2 > rc2 * (1.0 + 1e-5);
}

static int o_list(const o_system *sys, const double *q, const o_fix *fx, int i, double rc, o_nb *out,
                  int cap) {
    float rc2f = (float)(rc * rc);
    int n = 0;
    for (int j = 0; j < sys->n_atoms; ++j) {
        if (o_prefilter && j != i && o_beyond(sys, fx, i, j, rc * rc)) continue;
        for (int code = 0; code < 27; ++code) {
            int s[3] = {code % 3 - 1, (code / 3) % 3 - 1, code / 9 - 1};
            if (j == i && code == 13) continue;
            if (!o_member(sys, fx, i, j, s, rc2f, NULL)) continue;
            if (n >= cap) return -1;
            out[n].j = j;
            out[n].code = code;
            o_disp(sys, q, fx, i, j, s, out[n].d);
            out[n].r = sqrt(out[n].d[0] * out[n].d[0] + out[n].d[1] * out[n].d[1] + out[n].d[2] * out[n].d[2]);
            ++n;
        }
    }
    return n;
}

/* Exported: packed keys (j << 5 | code) per atom, row stride cap.  Returns 0 or
 * -1 when a row would exceed cap. */
int o_neighbors(const o_system *sys, const double *q, double rc, int32_t cap, int32_t *keys, int32_t *counts) {
    int N = sys->n_atoms;
    o_fix *fx = (o_fix *)malloc(sizeof(o_fix) * (size_t)N);
    o_nb *buf = (o_nb *)malloc(sizeof(o_nb) * (size_t)(cap > 0 ? cap : 1));
    o_fixpoint(sys, q, fx);
    int rc_ok = 0;
    for (int i = 0; i < N; ++i) {
        int n = o_list(sys, q, fx, i, rc, buf, cap);
        if (n < 0) { rc_ok = -1; counts[i] = -1; continue; }
        counts[i] = n;
        for (int k = 0; k < n; ++k) keys[(size_t)i * cap + k] = (buf[k].j << 5) | buf[k].code;
    }
    free(buf);
    free(fx);
    return rc_ok;
}

/* Exported for tests: fixed-point coordinates and image counts. */
void o_fixpoint_export(const o_system *sys, const double *q, uint32_t *u, int64_t *m) {
    o_fix *fx = (o_fix *)malloc(sizeof(o_fix) * (size_t)sys->n_atoms);
    o_fixpoint(sys, q, fx);
    for (int i = 0; i < sys->n_atoms; ++i)
        for (int a = 0; a < 3; ++a) { u[3 * i + a] = fx[i].u[a]; m[3 * i + a] = fx[i].m[a]; }
    free(fx);
}

/* ------------------------------------------------------------------------- */
/* Descriptors (the paper's force fields are external MLIPs; the synthetic     */
/* target follows the benchmark configuration: Gaussian radial basis times a  */
/* cosine cutoff, per neighbour species, plus Behler-type angular terms)       */
/* ------------------------------------------------------------------------- */

static double o_fc(double r, double rc) { return 0.5 * (cos(O_PI * r / rc) + 1.0); }
static double o_dfc(double r, double rc) { return -0.5 * O_PI / rc * sin(O_PI * r / rc); }

/* angular term a: zeta in {1,2,4,8} (slowest), lambda in {+1,-1}, eta in {0.005, 0.05} (fastest) */
static void o_ang_param(int a, double *zeta, double *lambda, double *eta) {
    static const double Z[4] = {1.0, 2.0, 4.0, 8.0};
    static const double E[2] = {0.005, 0.05};
    *zeta = Z[(a / 4) % 4];
    *lambda = ((a / 2) % 2) == 0 ? 1.0 : -1.0;
    *eta = E[a % 2];
}

/* Radial basis k of n_rbf: centre mu_k = k*rc/(n_rbf-1), width w = rc/(n_rbf-1). */
static void o_rbf(int k, int n_rbf, double rc, double r, double *g, double *dg) {
    double w = rc / (double)(n_rbf - 1);
    double mu = (double)k * w;
    double phi = exp(-(r - mu) * (r - mu) / (2.0 * w * w));
    double fc = o_fc(r, rc);
    *g = phi * fc;
    *dg = phi * (-(r - mu) / (w * w) * fc + o_dfc(r, rc));
}

/* One angular term T = 2^(1-zeta) (1 + lambda cos)^zeta exp(-eta (rp^2 + rq^2)) fc(rp) fc(rq)
 * and its gradients with respect to the displacement vectors dp, dq. */
static double o_ang_term(int a, double rc, const o_nb *P, const o_nb *Q, double gp[3], double gq[3]) {
    double zeta, lambda, eta;
    o_ang_param(a, &zeta, &lambda, &eta);
    double rp = P->r, rq = Q->r;
    double dot = P->d[0] * Q->d[0] + P->d[1] * Q->d[1] + P->d[2] * Q->d[2];
    double c = dot / (rp * rq);
    double base = 1.0 + lambda * c;
    double pw = pow(base, zeta);
    double pw1 = (zeta == 1.0) ? 1.0 : pow(base, zeta - 1.0);
    double ex = exp(-eta * (rp * rp + rq * rq));
    double fp = o_fc(rp, rc), fq = o_fc(rq, rc);
    double dfp = o_dfc(rp, rc), dfq = o_dfc(rq, rc);
    double pref = pow(2.0, 1.0 - zeta);
    double T = pref * pw * ex * fp * fq;
    if (gp && gq) {
        for (int x = 0; x < 3; ++x) {
            double dc_dp = Q->d[x] / (rp * rq) - c * P->d[x] / (rp * rp);
            double dc_dq = P->d[x] / (rp * rq) - c * Q->d[x] / (rq * rq);
            gp[x] = pref * (zeta * lambda * pw1 * dc_dp * ex * fp * fq + pw * ex * (-2.0 * eta * P->d[x]) * fp * fq +
                            pw * ex * dfp * (P->d[x] / rp) * fq);
            gq[x] = pref * (zeta * lambda * pw1 * dc_dq * ex * fp * fq + pw * ex * (-2.0 * eta * Q->d[x]) * fp * fq +
                            pw * ex * fp * dfq * (Q->d[x] / rq));
        }
    }
    return T;
}

/* Descriptor vector of one atom from its neighbour list (within desc_cutoff). */
static void o_descriptor(const o_system *sys, const o_potential *pot, int i, const o_nb *nb, int n, double *x) {
    int ns = sys->n_species, nr = pot->n_rbf, na = pot->n_ang;
    int d0 = o_input_dim(ns, nr, na);
    for (int f = 0; f < d0; ++f) x[f] = 0.0;
    for (int p = 0; p < n; ++p) {
        int sj = sys->species[nb[p].j];
        for (int k = 0; k < nr; ++k) {
            double g, dg;
            o_rbf(k, nr, pot->desc_cutoff, nb[p].r, &g, &dg);
            x[sj * nr + k] += g;
        }
    }
    for (int p = 0; p < n; ++p)
        for (int q2 = p + 1; q2 < n; ++q2)
            for (int a = 0; a < na; ++a) x[ns * nr + a] += o_ang_term(a, pot->desc_cutoff, &nb[p], &nb[q2], NULL, NULL);
    x[ns * nr + na + sys->species[i]] = 1.0;
}

/* ------------------------------------------------------------------------- */
/* Per-atom MLP: h_1 = W_1 x + b_1, a_l = SiLU(h_l), h_l = W_l a_{l-1} + b_l,  */
/* y = w_out . a_L + b_out, e = head_scale*tanh(y) or y.                       */
/* ------------------------------------------------------------------------- */

static double o_sigmoid(double h) { return 1.0 / (1.0 + exp(-h)); }
static double o_silu(double h) { return h * o_sigmoid(h); }
static double o_dsilu(double h) { double s = o_sigmoid(h); return s * (1.0 + h * (1.0 - s)); }
static double o_d2silu(double h) { double s = o_sigmoid(h); return s * (1.0 - s) * (2.0 + h * (1.0 - 2.0 * s)); }

typedef struct { const double *W, *b; int din, dout; } o_layer;

static void o_layers(const o_potential *pot, int d0, o_layer *L, const double **wout, const double **bout) {
    const double *w = pot->weights;
    int din = d0;
    for (int l = 0; l < pot->n_layers; ++l) {
        L[l].W = w; w += (size_t)pot->width * din;
        L[l].b = w; w += pot->width;
        L[l].din = din; L[l].dout = pot->width;
        din = pot->width;
    }
    *wout = w; w += pot->width;
    *bout = w;
}

/* Forward pass; h has n_layers*width entries (pre-activations); returns y. */
static double o_mlp_forward(const o_potential *pot, int d0, const double *x, double *h) {
    o_layer L[16];
    const double *wout, *bout;
    o_layers(pot, d0, L, &wout, &bout);
    int W = pot->width;
    double *a = (double *)malloc(sizeof(double) * (size_t)W);
    const double *in = x;
    for (int l = 0; l < pot->n_layers; ++l) {
        for (int o = 0; o < W; ++o) {
            double acc = L[l].b[o];
            for (int k = 0; k < L[l].din; ++k) acc += L[l].W[(size_t)o * L[l].din + k] * in[k];
            h[(size_t)l * W + o] = acc;
        }
        for (int o = 0; o < W; ++o) a[o] = o_silu(h[(size_t)l * W + o]);
        in = a;
    }
    double y = bout[0];
    for (int o = 0; o < W; ++o) y += wout[o] * in[o];
    free(a);
    return y;
}

static double o_head(const o_potential *pot, double y, double *dedy) {
    if (pot->head == O_HEAD_LINEAR) { *dedy = 1.0; return y; }
    double t = tanh(y);
    *dedy = pot->head_scale * (1.0 - t * t);
    return pot->head_scale * t;
}

/* Reverse pass: dE/dx given dE/dy and the stored pre-activations. */
static void o_mlp_backward(const o_potential *pot, int d0, const double *h, double dedy, double *dedx) {
    o_layer L[16];
    const double *wout, *bout;
    o_layers(pot, d0, L, &wout, &bout);
    int W = pot->width, nl = pot->n_layers;
    double *g = (double *)malloc(sizeof(double) * (size_t)W);
    double *gp = (double *)malloc(sizeof(double) * (size_t)(W > d0 ? W : d0));
    for (int o = 0; o < W; ++o) g[o] = dedy * wout[o] * o_dsilu(h[(size_t)(nl - 1) * W + o]);
    for (int l = nl - 1; l >= 0; --l) {
        int din = L[l].din;
        for (int k = 0; k < din; ++k) {
            double acc = 0.0;
            for (int o = 0; o < W; ++o) acc += L[l].W[(size_t)o * din + k] * g[o];
            gp[k] = acc;
        }
        if (l > 0) {
            for (int k = 0; k < din; ++k) g[k] = gp[k] * o_dsilu(h[(size_t)(l - 1) * W + k]);
        } else {
            for (int k = 0; k < din; ++k) dedx[k] = gp[k];
        }
    }
    free(g);
    free(gp);
}

/* ------------------------------------------------------------------------- */
/* Potential energy and forces                                                */
/* ------------------------------------------------------------------------- */

/* Threads of the loops over independent configurations (a window's K target
 * evaluations; o_eval_range); 1 (the default) runs them serially. */
static int o_threads = 1;

void o_set_threads(int32_t n) { o_threads = n > 0 ? n : 1; }

int o_get_threads(void) { return o_threads; }

#define O_NB_CAP 4096

static void o_lj_pair(double eps, double sig, double rc, double r, double *U, double *dU) {
    double sr6 = pow(sig / r, 6.0), sr12 = sr6 * sr6;
    double sc6 = pow(sig / rc, 6.0), sc12 = sc6 * sc6;
    *U = 4.0 * eps * (sr12 - sr6) - 4.0 * eps * (sc12 - sc6);
    *dU = -24.0 * eps / r * (2.0 * sr12 - sr6);
}

/* The terms of the energy whose centre atom i lies in [i0, i1): the LJ pairs
 * (i, j) (half of each pair's energy, the force on i) and e(x_i) with the
 * forces of its descriptor terms on i and its neighbours; F and E_atom are
 * accumulated, not cleared.  Over i in [0, N) this is every term of E. */
static double o_energy_forces_range(const o_system *sys, const o_potential *pot, const double *q, int i0, int i1,
                                    double *F, double *E_atom, double *X, double *dEdX) {
    int N = sys->n_atoms, ns = sys->n_species;
    double E = 0.0;
    o_fix *fx = (o_fix *)malloc(sizeof(o_fix) * (size_t)N);
    o_nb *nb = (o_nb *)malloc(sizeof(o_nb) * O_NB_CAP);
    o_fixpoint(sys, q, fx);
    int bad = 0;

    if (pot->lj_cutoff > 0.0) {
        for (int i = i0; i < i1; ++i) {
            int n = o_list(sys, q, fx, i, pot->lj_cutoff, nb, O_NB_CAP);
            if (n < 0) { bad = 1; break; }
            int si = sys->species[i];
            for (int p = 0; p < n; ++p) {
                int sj = sys->species[nb[p].j];
                double eps = sqrt(pot->lj_eps[si] * pot->lj_eps[sj]);      /* Lorentz-Berthelot */
                double sig = 0.5 * (pot->lj_sigma[si] + pot->lj_sigma[sj]);
                double U, dU;
                o_lj_pair(eps, sig, pot->lj_cutoff, nb[p].r, &U, &dU);
                E += 0.5 * U;
                if (E_atom) E_atom[i] += 0.5 * U;
                if (F) for (int a = 0; a < 3; ++a) F[3 * i + a] += dU * nb[p].d[a] / nb[p].r;
            }
        }
    }

    if (!bad && pot->n_layers > 0) {
        int d0 = o_input_dim(ns, pot->n_rbf, pot->n_ang);
        double *x = (double *)malloc(sizeof(double) * (size_t)d0);
        double *gx = (double *)malloc(sizeof(double) * (size_t)d0);
        double *h = (double *)malloc(sizeof(double) * (size_t)pot->n_layers * pot->width);
        for (int i = i0; i < i1 && !bad; ++i) {
            int n = o_list(sys, q, fx, i, pot->desc_cutoff, nb, O_NB_CAP);
            if (n < 0) { bad = 1; break; }
            o_descriptor(sys, pot, i, nb, n, x);
            double y = o_mlp_forward(pot, d0, x, h);
            double dedy;
            double e = o_head(pot, y, &dedy);
            E += e;
            if (E_atom) E_atom[i] += e;
            if (X) memcpy(X + (size_t)i * d0, x, sizeof(double) * (size_t)d0);
            if (!F && !dEdX) continue;
            o_mlp_backward(pot, d0, h, dedy, gx);
            if (dEdX) memcpy(dEdX + (size_t)i * d0, gx, sizeof(double) * (size_t)d0);
            if (!F) continue;
            int nr = pot->n_rbf;
            /* radial: x_{i,(s_j,k)} depends on r_ij; dr/dq_j = d/r, dr/dq_i = -d/r */
            for (int p = 0; p < n; ++p) {
                int sj = sys->species[nb[p].j];
                double c = 0.0;
                for (int k = 0; k < nr; ++k) {
                    double g, dg;
                    o_rbf(k, nr, pot->desc_cutoff, nb[p].r, &g, &dg);
                    c += gx[sj * nr + k] * dg;
                }
                for (int a = 0; a < 3; ++a) {
                    double v = c * nb[p].d[a] / nb[p].r;
                    F[3 * nb[p].j + a] -= v;
                    F[3 * i + a] += v;
                }
            }
            /* angular: T depends on d_p = q_jp - q_i and d_q = q_jq - q_i */
            for (int p = 0; p < n; ++p) {
                for (int q2 = p + 1; q2 < n; ++q2) {
                    for (int a = 0; a < pot->n_ang; ++a) {
                        double gp[3], gq[3];
                        o_ang_term(a, pot->desc_cutoff, &nb[p], &nb[q2], gp, gq);
                        double wgt = gx[ns * nr + a];
                        for (int x3 = 0; x3 < 3; ++x3) {
                            F[3 * nb[p].j + x3] -= wgt * gp[x3];
                            F[3 * nb[q2].j + x3] -= wgt * gq[x3];
                            F[3 * i + x3] += wgt * (gp[x3] + gq[x3]);
                        }
                    }
                }
            }
        }
        free(x);
        free(gx);
        free(h);
    }
    free(nb);
    free(fx);
    return bad ? NAN : E;
}

/* E = sum of LJ (shifted, all periodic images within cutoff) + sum_i e(x_i)
 * + harmonic tether.  F = -dE/dq (+ the optional non-conservative shear field).
 * Optional outputs: per-atom energies, descriptors X [N][d0], dE/dX [N][d0].
 * Returns the total energy, or NAN when a neighbour list overflows. */
double o_energy_forces(const o_system *sys, const o_potential *pot, const double *q, double *F, double *E_atom,
                       double *X, double *dEdX) {
    int N = sys->n_atoms;
    if (F) for (int k = 0; k < 3 * N; ++k) F[k] = 0.0;
    if (E_atom) for (int i = 0; i < N; ++i) E_atom[i] = 0.0;
    double E = o_energy_forces_range(sys, pot, q, 0, N, F, E_atom, X, dEdX);
    int bad = isnan(E);

    if (!bad && pot->k_harm > 0.0) {
        for (int k = 0; k < 3 * N; ++k) {
            double dq = q[k] - pot->q_ref[k];
            E += 0.5 * pot->k_harm * dq * dq;
            if (E_atom) E_atom[k / 3] += 0.5 * pot->k_harm * dq * dq;
            if (F) F[k] -= pot->k_harm * dq;
        }
    }
    if (!bad && pot->shear != 0.0 && F) {
        for (int i = 0; i < N; ++i) F[3 * i + 0] += pot->shear * sin(2.0 * O_PI * q[3 * i + 1] / sys->box[1]);
    }
    return bad ? NAN : E;
}

/* The centre-atom terms [i0, i1) of the energy and forces (LJ + MLP
 * potentials; no tether or shear field) of C configurations q [C][N][3]: F
 * [C][N][3] and E [C] are cleared, then receive those terms.  The C
 * configurations run on o_set_threads() threads, one configuration each, as
 * in the window's verification loop.  Summed over the ranges of a partition
 * of [0, N), this is o_energy_forces.  Used to time a bounded slice of an
 * evaluation too large to run whole.  Returns 0, or -1 on a list overflow. */
int o_eval_range(const o_system *sys, const o_potential *pot, int32_t C, const double *q, int32_t i0, int32_t i1,
                 double *F, double *E) {
    int N = sys->n_atoms;
    if (i0 < 0 || i1 > N || i0 > i1 || C < 1) return -2;
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) num_threads(o_threads) if (o_threads > 1) reduction(| : bad)
    for (int c = 0; c < C; ++c) {
        double *Fc = F + (size_t)c * 3 * N;
        for (int k = 0; k < 3 * N; ++k) Fc[k] = 0.0;
        E[c] = o_energy_forces_range(sys, pot, q + (size_t)c * 3 * N, i0, i1, Fc, NULL, NULL, NULL);
        bad |= isnan(E[c]);
    }
    return bad ? -1 : 0;
}

/* Forces on selected atoms only, one atom at a time, for systems too large
 * for a full pass: F_a = -dE/dq_a collects the LJ pairs of a and, for every
 * atom i whose descriptor depends on q_a (i = a and the descriptor neighbours
 * of a), the terms of E_i that involve a.  Same definitions as
 * o_energy_forces (LJ + MLP potentials; no tether or shear field).
 * F_out: [n_sel][3].  Returns 0, or -1 when a neighbour list overflows. */
int o_forces_subset(const o_system *sys, const o_potential *pot, const double *q, int32_t n_sel,
                    const int32_t *sel, double *F_out) {
    int N = sys->n_atoms, ns = sys->n_species;
    for (int t = 0; t < n_sel; ++t)
        if (sel[t] < 0 || sel[t] >= N) return -2;
    o_fix *fx = (o_fix *)malloc(sizeof(o_fix) * (size_t)N);
    o_nb *nb = (o_nb *)malloc(sizeof(o_nb) * O_NB_CAP);
    o_nb *nbi = (o_nb *)malloc(sizeof(o_nb) * O_NB_CAP);
    o_fixpoint(sys, q, fx);
    int d0 = pot->n_layers > 0 ? o_input_dim(ns, pot->n_rbf, pot->n_ang) : 1;
    double *x = (double *)malloc(sizeof(double) * (size_t)d0);
    double *gx = (double *)malloc(sizeof(double) * (size_t)d0);
    double *h = (double *)malloc(sizeof(double) * (size_t)(pot->n_layers > 0 ? pot->n_layers * pot->width : 1));
    int ret = 0;
    for (int t = 0; t < n_sel && ret == 0; ++t) {
        int a = sel[t];
        double Fa[3] = {0.0, 0.0, 0.0};
        if (pot->lj_cutoff > 0.0) {
            int n = o_list(sys, q, fx, a, pot->lj_cutoff, nb, O_NB_CAP);
            if (n < 0) { ret = -1; break; }
            int sa = sys->species[a];
            for (int p = 0; p < n; ++p) {
                int sj = sys->species[nb[p].j];
                double eps = sqrt(pot->lj_eps[sa] * pot->lj_eps[sj]);
                double sig = 0.5 * (pot->lj_sigma[sa] + pot->lj_sigma[sj]);
                double U, dU;
                o_lj_pair(eps, sig, pot->lj_cutoff, nb[p].r, &U, &dU);
                for (int c = 0; c < 3; ++c) Fa[c] += dU * nb[p].d[c] / nb[p].r;
            }
        }
        if (pot->n_layers > 0) {
            int na = o_list(sys, q, fx, a, pot->desc_cutoff, nb, O_NB_CAP);
            if (na < 0) { ret = -1; break; }
            int nr = pot->n_rbf;
            /* candidates i: a itself and its descriptor neighbours (several images of one atom count once) */
            for (int cnd = -1; cnd < na; ++cnd) {
                int i = cnd < 0 ? a : nb[cnd].j;
                int dup = 0;
                if (cnd >= 0) {
                    if (i == a) dup = 1;
                    for (int e = 0; e < cnd && !dup; ++e) dup = (nb[e].j == i);
                }
                if (dup) continue;
                int n = o_list(sys, q, fx, i, pot->desc_cutoff, nbi, O_NB_CAP);
                if (n < 0) { ret = -1; break; }
                o_descriptor(sys, pot, i, nbi, n, x);
                double y = o_mlp_forward(pot, d0, x, h);
                double dedy;
                o_head(pot, y, &dedy);
                o_mlp_backward(pot, d0, h, dedy, gx);
                /* -dE_i/dq_a: radial and angular terms of E_i through the displacement vectors */
                for (int p = 0; p < n; ++p) {
                    int sj = sys->species[nbi[p].j];
                    double cr = 0.0;
                    for (int k = 0; k < nr; ++k) {
                        double g, dg;
                        o_rbf(k, nr, pot->desc_cutoff, nbi[p].r, &g, &dg);
                        cr += gx[sj * nr + k] * dg;
                    }
                    double coef = (nbi[p].j == a ? -1.0 : 0.0) + (i == a ? 1.0 : 0.0);
                    for (int c = 0; c < 3; ++c) Fa[c] += coef * cr * nbi[p].d[c] / nbi[p].r;
                }
                for (int p = 0; p < n; ++p)
                    for (int q2 = p + 1; q2 < n; ++q2)
                        for (int an = 0; an < pot->n_ang; ++an) {
                            double gp[3], gq[3];
                            o_ang_term(an, pot->desc_cutoff, &nbi[p], &nbi[q2], gp, gq);
                            double wgt = gx[ns * nr + an];
                            double cp = (nbi[p].j == a ? -1.0 : 0.0) + (i == a ? 1.0 : 0.0);
                            double cq = (nbi[q2].j == a ? -1.0 : 0.0) + (i == a ? 1.0 : 0.0);
                            for (int c = 0; c < 3; ++c) Fa[c] += wgt * (cp * gp[c] + cq * gq[c]);
                        }
            }
        }
        for (int c = 0; c < 3; ++c) F_out[3 * t + c] = Fa[c];
    }
    free(x); free(gx); free(h); free(nb); free(nbi); free(fx);
    return ret;
}

/* ------------------------------------------------------------------------- */
/* ABOBA (Eq. 2) and the BOB Gaussian (Eq. 4)                                 */
/* ------------------------------------------------------------------------- */

typedef struct {
    double c1;     /* exp(-gamma dt) */
    double h;      /* dt / 2 */
    double aF;     /* (1 + c1) (dt/2) kappa: force -> mean momentum shift */
    double *hm;    /* per species (dt/2)/m */
    double *sig;   /* per species sqrt(m kB T kappa (1 - exp(-2 gamma dt))) */
    /* OBABO (App. E) */
    int obabo;
    double ch;     /* exp(-gamma dt/2): friction of a half-step O */
    double bF;     /* (dt/2) kappa: one B half-step kick per unit force */
    double *hmf;   /* per species dt/m: the full-step A of the staggered frame */
    double *sigh;  /* per species sqrt(m kB T kappa (1 - exp(-gamma dt))): half-step O noise, Sigma_1/2 */
} o_coef;

static void o_coef_init(const o_system *sys, const o_params *prm, o_coef *c) {
    double kappa = o_kappa(), kB = o_kboltz();
    c->c1 = exp(-prm->gamma * prm->dt);
    c->h = 0.5 * prm->dt;
    c->aF = (1.0 + c->c1) * c->h * kappa;
    c->hm = (double *)malloc(sizeof(double) * (size_t)sys->n_species);
    c->sig = (double *)malloc(sizeof(double) * (size_t)sys->n_species);
    c->hmf = (double *)malloc(sizeof(double) * (size_t)sys->n_species);
    c->sigh = (double *)malloc(sizeof(double) * (size_t)sys->n_species);
    c->obabo = prm->integrator == O_OBABO;
    c->ch = exp(-0.5 * prm->gamma * prm->dt);
    c->bF = c->h * kappa;
    double one_minus = -expm1(-2.0 * prm->gamma * prm->dt);
    double one_minus_half = -expm1(-prm->gamma * prm->dt);
    for (int s = 0; s < sys->n_species; ++s) {
        double m = sys->species_mass[s];
        c->hm[s] = c->h / m;
        c->sig[s] = sqrt(m * kB * prm->temperature * kappa * one_minus);
        c->hmf[s] = prm->dt / m;
        c->sigh[s] = sqrt(m * kB * prm->temperature * kappa * one_minus_half);
    }
}
static void o_coef_free(o_coef *c) { free(c->hm); free(c->sig); free(c->hmf); free(c->sigh); }

/* Exported so tests can see the coefficients the oracle uses. */
void o_coefficients(const o_system *sys, const o_params *prm, double *c1, double *aF, double *hm, double *sig) {
    o_coef c;
    o_coef_init(sys, prm, &c);
    *c1 = c.c1;
    *aF = c.aF;
    for (int s = 0; s < sys->n_species; ++s) { hm[s] = c.hm[s]; sig[s] = c.sig[s]; }
    o_coef_free(&c);
}

/* Maxwell-Boltzmann momenta p = sqrt(m kB T kappa) xi with xi from stream 2, step 0. */
void o_mb_momenta(const o_system *sys, const o_params *prm, double *p) {
    double kappa = o_kappa(), kB = o_kboltz();
    for (int i = 0; i < sys->n_atoms; ++i) {
        double xi[3];
        o_normals(prm->seed, 0, (uint32_t)i, 2u, xi);
        double sd = sqrt(sys->species_mass[sys->species[i]] * kB * prm->temperature * kappa);
        for (int a = 0; a < 3; ++a) p[3 * i + a] = sd * xi[a];
    }
}

/* One ABOBA step (Eq. 2) producing step index n with force field pot, written
 * as A, then the BOB Gaussian draw of Eq. 4, then A.  dF (may be NULL) is
 * added to the force before forming the mean (speculative error correction).
 * Outputs the half-step positions, the raw force, the mean and the new state. */
static int o_aboba(const o_system *sys, const o_potential *pot, const o_params *prm, const o_coef *c, uint64_t n,
                   const double *q, const double *p, const double *dF, double *qmid, double *Fraw, double *mu,
                   double *q_new, double *p_new) {
    int N = sys->n_atoms;
    for (int i = 0; i < N; ++i) {
        /* A: half step of ABOBA, or the full step of the staggered OBABO frame (App. E) */
        double hm = c->obabo ? c->hmf[sys->species[i]] : c->hm[sys->species[i]];
        for (int a = 0; a < 3; ++a) qmid[3 * i + a] = q[3 * i + a] + p[3 * i + a] * hm;
    }
    double E = o_energy_forces(sys, pot, qmid, Fraw, NULL, NULL, NULL);
    if (isnan(E)) return -1;
    for (int i = 0; i < N; ++i) {
        double xi[3];
        o_normals(prm->seed, n, (uint32_t)i, 0u, xi);
        int s = sys->species[i];
        for (int a = 0; a < 3; ++a) {
            int k = 3 * i + a;
            double Fk = dF ? Fraw[k] + dF[k] : Fraw[k];
            mu[k] = c->c1 * p[k] + c->aF * Fk;          /* BOB mean, Eq. 4 */
            p_new[k] = mu[k] + c->sig[s] * xi[a];         /* BOB draw */
            q_new[k] = c->obabo ? qmid[k] : qmid[k] + p_new[k] * c->hm[s];   /* A (ABOBA); none (staggered OBABO) */
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* reflectionVerify (Eq. 5) on the momenta after BOB, then the shared A map    */
/* (Thm 3.1, Alg. 2 verify_step).                                             */
/* ------------------------------------------------------------------------- */

typedef struct {
    int accept;
    double log_ratio;   /* log N(p~; <p>, S) - log N(p~; <p~>, S) */
    double log_u;
    double delta_norm;  /* Mahalanobis distance |delta| */
} o_verdict;

static o_verdict o_reflection_verify(const o_system *sys, const o_coef *c, double u, const double *p_draft,
                                     const double *mu_draft, const double *mu_target, const double *qmid,
                                     double *q_out, double *p_out) {
    int D = 3 * sys->n_atoms;
    double lr = 0.0, zd = 0.0, dd = 0.0;
    for (int k = 0; k < D; ++k) {
        double sg = c->sig[sys->species[k / 3]];
        double z = (p_draft[k] - mu_draft[k]) / sg;        /* z = S^-1/2 (p~ - <p~>) */
        double e = (p_draft[k] - mu_target[k]) / sg;       /* S^-1/2 (p~ - <p>) */
        double dl = (mu_draft[k] - mu_target[k]) / sg;     /* delta = S^-1/2 (<p~> - <p>) */
        lr += -0.5 * e * e + 0.5 * z * z;
        zd += z * dl;
        dd += dl * dl;
    }
    o_verdict v;
    v.log_ratio = lr;
    v.log_u = log(u);
    v.delta_norm = sqrt(dd);
    /* accept iff u <= min(1, ratio), compared in log space */
    v.accept = (dd == 0.0) || (v.log_u <= (lr < 0.0 ? lr : 0.0));
    for (int k = 0; k < D; ++k) {
        int s = sys->species[k / 3];
        if (v.accept) {
            p_out[k] = p_draft[k];
        } else {
            double sg = c->sig[s];
            double z = (p_draft[k] - mu_draft[k]) / sg;
            double dl = (mu_draft[k] - mu_target[k]) / sg;
            p_out[k] = mu_target[k] + sg * (z - 2.0 * (zd / dd) * dl);   /* Householder reflection */
        }
        q_out[k] = c->obabo ? qmid[k] : qmid[k] + p_out[k] * c->hm[s];   /* map g = A (ABOBA), id (OBABO) */
    }
    return v;
}

/* Exported 1-D/generic transport for tests: given the draft momentum, both
 * means, per-component sigma and u, returns the accept flag and writes p. */
int o_transport_terms(int32_t D, const double *sig, double u, const double *p_draft, const double *mu_draft,
                      const double *mu_target, double *p_out, double *log_ratio, double *zdelta, double *deltadelta);

int o_transport(int32_t D, const double *sig, double u, const double *p_draft, const double *mu_draft,
                const double *mu_target, double *p_out, double *log_ratio) {
    return o_transport_terms(D, sig, u, p_draft, mu_draft, mu_target, p_out, log_ratio, NULL, NULL);
}

/* reflectionVerify as above; also returns z.delta and delta.delta (either
 * pointer may be NULL), the two sums Eq. 5 and Eq. 6 are built from. */
int o_transport_terms(int32_t D, const double *sig, double u, const double *p_draft, const double *mu_draft,
                      const double *mu_target, double *p_out, double *log_ratio, double *zdelta, double *deltadelta) {
    double lr = 0.0, zd = 0.0, dd = 0.0;
    for (int k = 0; k < D; ++k) {
        double z = (p_draft[k] - mu_draft[k]) / sig[k];
        double e = (p_draft[k] - mu_target[k]) / sig[k];
        double dl = (mu_draft[k] - mu_target[k]) / sig[k];
        lr += -0.5 * e * e + 0.5 * z * z;
        zd += z * dl;
        dd += dl * dl;
    }
    int acc = (dd == 0.0) || (log(u) <= (lr < 0.0 ? lr : 0.0));
    for (int k = 0; k < D; ++k) {
        if (acc) p_out[k] = p_draft[k];
        else {
            double z = (p_draft[k] - mu_draft[k]) / sig[k];
            double dl = (mu_draft[k] - mu_target[k]) / sig[k];
            p_out[k] = mu_target[k] + sig[k] * (z - 2.0 * (zd / dd) * dl);
        }
    }
    if (log_ratio) *log_ratio = lr;
    if (zdelta) *zdelta = zd;
    if (deltadelta) *deltadelta = dd;
    return acc;
}

/* ------------------------------------------------------------------------- */
/* OBABO through the staggered frame (App. E)                                  */
/* ------------------------------------------------------------------------- */

/* The OBABO output momentum of staggered step n (App. E): with the staggered
 * momenta p_prev (before) and p_new (after) and the step's target force F,
 * p_in = p_prev + (dt/2) kappa F, and w = Sigma_1/2^-1/2 (p_new - c1 p_prev -
 * (1 + c1) (dt/2) kappa F) fixes e^(-gamma dt/2) xi1 + xi2.  xi1 is drawn from
 * its conditional law N(e^(-gamma dt/2) w / (1 + c1), 1 / (1 + c1)) with the
 * standard normal eta of stream 3 at step n, and p_mid = e^(-gamma dt/2) p_in +
 * Sigma_1/2^1/2 xi1. */
static void o_obabo_recover(const o_system *sys, const o_coef *c, uint64_t seed, uint64_t n, const double *p_prev,
                            const double *F, const double *p_new, double *p_mid) {
    double a = c->ch / (1.0 + c->c1), b = sqrt(1.0 / (1.0 + c->c1));
    for (int i = 0; i < sys->n_atoms; ++i) {
        double eta[3];
        o_normals(seed, n, (uint32_t)i, 3u, eta);
        double sh = c->sigh[sys->species[i]];
        for (int x = 0; x < 3; ++x) {
            int k = 3 * i + x;
            double p_in = p_prev[k] + c->bF * F[k];
            double w = (p_new[k] - c->c1 * p_prev[k] - c->aF * F[k]) / sh;
            double xi1 = a * w + b * eta[x];
            p_mid[k] = c->ch * p_in + sh * xi1;
        }
    }
}

void o_obabo_output(const o_system *sys, const o_params *prm, int64_t n, const double *p_prev, const double *F,
                    const double *p_new, double *p_mid) {
    o_coef c;
    o_coef_init(sys, prm, &c);
    o_obabo_recover(sys, &c, prm->seed, (uint64_t)n, p_prev, F, p_new, p_mid);
    o_coef_free(&c);
}

/* Enters the staggered frame from an OBABO state (q, p) at step index n: the
 * leading O half-step (noise of stream 4 at n) and B half-step at q,
 * p <- e^(-gamma dt/2) p + Sigma_1/2^1/2 xi + (dt/2) kappa F(q). */
int o_obabo_enter(const o_system *sys, const o_potential *target, const o_params *prm, int64_t n, const double *q,
                  double *p) {
    int D = 3 * sys->n_atoms;
    o_coef c;
    o_coef_init(sys, prm, &c);
    double *F = (double *)malloc(sizeof(double) * (size_t)D);
    double E = o_energy_forces(sys, target, q, F, NULL, NULL, NULL);
    int ret = isnan(E) ? -1 : 0;
    for (int i = 0; i < sys->n_atoms && ret == 0; ++i) {
        double xi[3];
        o_normals(prm->seed, (uint64_t)n, (uint32_t)i, 4u, xi);
        double sh = c.sigh[sys->species[i]];
        for (int x = 0; x < 3; ++x) {
            int k = 3 * i + x;
            p[k] = (c.ch * p[k] + sh * xi[x]) + c.bF * F[k];
        }
    }
    free(F);
    o_coef_free(&c);
    return ret;
}

/* The OBABO integrator written out literally (O, B, A, B, O per step, noise of
 * streams 5 and 6 at the produced step index), for distribution tests of the
 * staggered construction.  traj as in o_plain_run. */
int o_obabo_literal(const o_system *sys, const o_potential *pot, const o_params *prm, int64_t n_steps, double *q,
                    double *p, int64_t *step, double *traj_q, double *traj_p) {
    int N = sys->n_atoms, D = 3 * N;
    o_coef c;
    o_coef_init(sys, prm, &c);
    double *F = (double *)malloc(sizeof(double) * (size_t)D);
    int ret = 0;
    if (isnan(o_energy_forces(sys, pot, q, F, NULL, NULL, NULL))) ret = -1;
    for (int64_t t = 0; t < n_steps && ret == 0; ++t) {
        uint64_t n = (uint64_t)(*step + 1);
        for (int i = 0; i < N; ++i) {
            double xi[3];
            o_normals(prm->seed, n, (uint32_t)i, 5u, xi);
            int s = sys->species[i];
            for (int x = 0; x < 3; ++x) {
                int k = 3 * i + x;
                p[k] = c.ch * p[k] + c.sigh[s] * xi[x];   /* O */
                p[k] += c.bF * F[k];                      /* B */
                q[k] += c.hmf[s] * p[k];                  /* A, full step */
            }
        }
        if (isnan(o_energy_forces(sys, pot, q, F, NULL, NULL, NULL))) { ret = -1; break; }
        for (int i = 0; i < N; ++i) {
            double xi[3];
            o_normals(prm->seed, n, (uint32_t)i, 6u, xi);
            int s = sys->species[i];
            for (int x = 0; x < 3; ++x) {
                int k = 3 * i + x;
                p[k] += c.bF * F[k];                      /* B */
                p[k] = c.ch * p[k] + c.sigh[s] * xi[x];   /* O */
            }
        }
        *step += 1;
        if (traj_q) memcpy(traj_q + (size_t)t * D, q, sizeof(double) * (size_t)D);
        if (traj_p) memcpy(traj_p + (size_t)t * D, p, sizeof(double) * (size_t)D);
    }
    free(F);
    o_coef_free(&c);
    return ret;
}

/* ------------------------------------------------------------------------- */
/* One synchronous speculative window (Alg. 1 with lookahead L = K), ABOBA     */
/* draft_step / verify_step of Alg. 2, optional error correction (Alg. 3).    */
/* ------------------------------------------------------------------------- */

/* Drafts K steps from (q, p) at step index n0, verifies each against the target,
 * commits the accepted prefix plus the first rejected (reflected) step, at most
 * max_commit steps, and overwrites (q, p) with the last committed state.
 * ec_dF, when not NULL, is the error-correction cache: added to the draft
 * force, and replaced on commit by F - F~raw of the last committed step.
 * Window arrays (each may be NULL): [K][3N] half-step positions, draft
 * momenta, draft means, raw draft forces, target forces; [K] log ratio, log u,
 * |delta|, accept flag.  Returns the number of committed steps, or < 0. */
int o_lsd_window(const o_system *sys, const o_potential *draft, const o_potential *target, const o_params *prm,
                 int64_t n0, int32_t K, int32_t max_commit, double *q, double *p, double *ec_dF, double *w_qmid,
                 double *w_pdraft, double *w_mudraft, double *w_Fdraft, double *w_Ftarget, double *w_logr,
                 double *w_logu, double *w_dnorm, int32_t *w_accept, double *p_obabo) {
    int N = sys->n_atoms, D = 3 * N;
    o_coef c;
    o_coef_init(sys, prm, &c);
    size_t KD = (size_t)K * D;
    double *qmid = (double *)malloc(sizeof(double) * KD);
    double *pd = (double *)malloc(sizeof(double) * KD);
    double *qd = (double *)malloc(sizeof(double) * KD);
    double *mud = (double *)malloc(sizeof(double) * KD);
    double *Fd = (double *)malloc(sizeof(double) * KD);
    double *Ft = (double *)malloc(sizeof(double) * KD);
    double *mut = (double *)malloc(sizeof(double) * (size_t)D);
    double *qx = (double *)malloc(sizeof(double) * KD);
    double *px = (double *)malloc(sizeof(double) * KD);
    int *acc = (int *)malloc(sizeof(int) * (size_t)K);
    int ret = 0;

    /* draft, serial in j (Alg. 1 first loop) */
    for (int j = 0; j < K && ret == 0; ++j) {
        const double *qin = (j == 0) ? q : qd + (size_t)(j - 1) * D;
        const double *pin = (j == 0) ? p : pd + (size_t)(j - 1) * D;
        if (o_aboba(sys, draft, prm, &c, (uint64_t)(n0 + j + 1), qin, pin, ec_dF, qmid + (size_t)j * D,
                    Fd + (size_t)j * D, mud + (size_t)j * D, qd + (size_t)j * D, pd + (size_t)j * D) != 0)
            ret = -1;
    }
    /* verify every window step (Alg. 1 parallel loop): the K target evaluations
     * are independent, so with o_set_threads(n > 1) they run on n threads, each
     * step's arithmetic unchanged (same result as one thread, bit for bit) */
    double *Et = (double *)malloc(sizeof(double) * (size_t)K);
    if (ret == 0) {
#pragma omp parallel for schedule(dynamic, 1) num_threads(o_threads) if (o_threads > 1)
        for (int j = 0; j < K; ++j)
            Et[j] = o_energy_forces(sys, target, qmid + (size_t)j * D, Ft + (size_t)j * D, NULL, NULL, NULL);
    }
    for (int j = 0; j < K && ret == 0; ++j) {
        const double *pin = (j == 0) ? p : pd + (size_t)(j - 1) * D;
        if (isnan(Et[j])) { ret = -1; break; }
        for (int k = 0; k < D; ++k) mut[k] = c.c1 * pin[k] + c.aF * Ft[(size_t)j * D + k];   /* <p>, Eq. 4 */
        double u = o_uniform(prm->seed, (uint64_t)(n0 + j + 1));
        o_verdict v = o_reflection_verify(sys, &c, u, pd + (size_t)j * D, mud + (size_t)j * D, mut,
                                          qmid + (size_t)j * D, qx + (size_t)j * D, px + (size_t)j * D);
        acc[j] = v.accept;
        if (w_logr) w_logr[j] = v.log_ratio;
        if (w_logu) w_logu[j] = v.log_u;
        if (w_dnorm) w_dnorm[j] = v.delta_norm;
        if (w_accept) w_accept[j] = v.accept;
    }
    int n_commit = 0;
    if (ret == 0) {
        /* l = first rejected step (1-based), else K; commit x_1..x_l */
        int l = K;
        for (int j = 0; j < K; ++j) if (!acc[j]) { l = j + 1; break; }
        n_commit = l < max_commit ? l : max_commit;
        int last = n_commit - 1;
        if (c.obabo && p_obabo) {
            /* the OBABO output of the last committed step, from its staggered momenta and target force */
            const double *pprev = last == 0 ? p : pd + (size_t)(last - 1) * D;
            o_obabo_recover(sys, &c, prm->seed, (uint64_t)(n0 + last + 1), pprev, Ft + (size_t)last * D,
                            px + (size_t)last * D, p_obabo);
        }
        memcpy(q, qx + (size_t)last * D, sizeof(double) * (size_t)D);
        memcpy(p, px + (size_t)last * D, sizeof(double) * (size_t)D);
        if (ec_dF)
            for (int k = 0; k < D; ++k) ec_dF[k] = Ft[(size_t)last * D + k] - Fd[(size_t)last * D + k];
        if (w_qmid) memcpy(w_qmid, qmid, sizeof(double) * KD);
        if (w_pdraft) memcpy(w_pdraft, pd, sizeof(double) * KD);
        if (w_mudraft) memcpy(w_mudraft, mud, sizeof(double) * KD);
        if (w_Fdraft) memcpy(w_Fdraft, Fd, sizeof(double) * KD);
        if (w_Ftarget) memcpy(w_Ftarget, Ft, sizeof(double) * KD);
    }
    free(qmid); free(pd); free(qd); free(mud); free(Fd); free(Ft); free(mut); free(qx); free(px); free(acc); free(Et);
    o_coef_free(&c);
    return ret == 0 ? n_commit : ret;
}

/* Runs LSD windows until n_steps steps are committed, from step index *step.
 * traj_q / traj_p (may be NULL): [n_steps][3N] committed states in order
 * (for committed steps other than each window's last, the state is the
 * accepted draft, which the window arrays give).  stats (may be NULL), 6
 * entries: windows, committed, rejected, sum of predicted rejection
 * erf(|delta|/sqrt 8) over committed steps, sum of |delta| over committed
 * steps, verified steps.  Returns 0 or < 0. */
int o_lsd_run(const o_system *sys, const o_potential *draft, const o_potential *target, const o_params *prm,
              int64_t n_steps, int32_t K, int32_t use_ec, double *q, double *p, int64_t *step, double *traj_q,
              double *traj_p, double *stats, double *p_obabo) {
    int N = sys->n_atoms, D = 3 * N;
    size_t KD = (size_t)K * D;
    double *pd = (double *)malloc(sizeof(double) * KD);
    double *qmid = (double *)malloc(sizeof(double) * KD);
    double *logr = (double *)malloc(sizeof(double) * (size_t)K);
    double *logu = (double *)malloc(sizeof(double) * (size_t)K);
    double *dn = (double *)malloc(sizeof(double) * (size_t)K);
    int32_t *acc = (int32_t *)malloc(sizeof(int32_t) * (size_t)K);
    double *dF = use_ec ? (double *)calloc((size_t)D, sizeof(double)) : NULL;
    double *Ft = (double *)malloc(sizeof(double) * KD);
    double *pbase = (double *)malloc(sizeof(double) * (size_t)D);
    double *pout = (double *)malloc(sizeof(double) * (size_t)D);
    o_coef c;
    o_coef_init(sys, prm, &c);
    double st[6] = {0, 0, 0, 0, 0, 0};
    int64_t done = 0;
    int ret = 0;
    while (done < n_steps) {
        int64_t rem = n_steps - done;
        int32_t kk = (int32_t)(rem < K ? rem : K);
        memcpy(pbase, p, sizeof(double) * (size_t)D);
        int nc = o_lsd_window(sys, draft, target, prm, *step, kk, kk, q, p, dF, qmid, pd, NULL, NULL, Ft, logr,
                              logu, dn, acc, pout);
        if (nc < 0) { ret = nc; break; }
        st[0] += 1; st[1] += nc; st[5] += kk;
        for (int j = 0; j < nc; ++j) {
            st[3] += erf(dn[j] / sqrt(8.0));
            st[4] += dn[j];
            if (!acc[j]) st[2] += 1;
            if ((traj_q || traj_p) && c.obabo) {
                /* OBABO outputs: positions of the staggered states, recovered momenta */
                size_t off = (size_t)(done + j) * D;
                const double *pprev = j == 0 ? pbase : pd + (size_t)(j - 1) * D;
                const double *pnew = j == nc - 1 ? p : pd + (size_t)j * D;
                if (traj_q) memcpy(traj_q + off, j == nc - 1 ? q : qmid + (size_t)j * D, sizeof(double) * (size_t)D);
                if (traj_p)
                    o_obabo_recover(sys, &c, prm->seed, (uint64_t)(*step + j + 1), pprev, Ft + (size_t)j * D, pnew,
                                    traj_p + off);
            } else if (traj_q || traj_p) {
                size_t off = (size_t)(done + j) * D;
                if (j == nc - 1) {
                    if (traj_q) memcpy(traj_q + off, q, sizeof(double) * (size_t)D);
                    if (traj_p) memcpy(traj_p + off, p, sizeof(double) * (size_t)D);
                } else {
                    for (int k = 0; k < D; ++k) {
                        double pk = pd[(size_t)j * D + k];
                        if (traj_p) traj_p[off + k] = pk;
                        if (traj_q) traj_q[off + k] = qmid[(size_t)j * D + k] + pk * c.hm[sys->species[k / 3]];
                    }
                }
            }
        }
        done += nc;
        *step += nc;
        if (p_obabo && c.obabo) memcpy(p_obabo, pout, sizeof(double) * (size_t)D);
    }
    if (stats) memcpy(stats, st, sizeof(st));
    free(pd); free(qmid); free(logr); free(logu); free(dn); free(acc); free(dF); free(Ft); free(pbase); free(pout);
    o_coef_free(&c);
    return ret;
}

/* Plain target Langevin: n_steps ABOBA steps with the target force field, noise
 * keyed by the step index exactly as in the draft.  traj as in o_lsd_run. */
int o_plain_run(const o_system *sys, const o_potential *target, const o_params *prm, int64_t n_steps, double *q,
                double *p, int64_t *step, double *traj_q, double *traj_p, double *p_obabo) {
    int D = 3 * sys->n_atoms;
    o_coef c;
    o_coef_init(sys, prm, &c);
    double *qmid = (double *)malloc(sizeof(double) * (size_t)D);
    double *F = (double *)malloc(sizeof(double) * (size_t)D);
    double *mu = (double *)malloc(sizeof(double) * (size_t)D);
    double *qn = (double *)malloc(sizeof(double) * (size_t)D);
    double *pn = (double *)malloc(sizeof(double) * (size_t)D);
    double *pm = (double *)malloc(sizeof(double) * (size_t)D);
    int ret = 0;
    for (int64_t t = 0; t < n_steps; ++t) {
        if (o_aboba(sys, target, prm, &c, (uint64_t)(*step + 1), q, p, NULL, qmid, F, mu, qn, pn) != 0) {
            ret = -1;
            break;
        }
        if (c.obabo) {   /* OBABO output of this step (App. E) */
            o_obabo_recover(sys, &c, prm->seed, (uint64_t)(*step + 1), p, F, pn, pm);
            if (p_obabo) memcpy(p_obabo, pm, sizeof(double) * (size_t)D);
        }
        memcpy(q, qn, sizeof(double) * (size_t)D);
        memcpy(p, pn, sizeof(double) * (size_t)D);
        *step += 1;
        if (traj_q) memcpy(traj_q + (size_t)t * D, q, sizeof(double) * (size_t)D);
        if (traj_p) memcpy(traj_p + (size_t)t * D, c.obabo ? pm : p, sizeof(double) * (size_t)D);
    }
    free(qmid); free(F); free(mu); free(qn); free(pn); free(pm);
    o_coef_free(&c);
    return ret;
}

/* ------------------------------------------------------------------------- */
/* Force matching of a learned draft (linear head), with its exact gradient    */
/* ------------------------------------------------------------------------- */
/* Loss L = (1/(n_frames*3N)) sum_frames |F~(q) - F*|^2 where F~ = -dE~/dq and
 * E~ = LJ + sum_i y(x_i; theta).  With r = F~ - F* and v_i = (dx_i/dq) r (the
 * descriptor JVP along the residual), dL/dtheta = -(2/(n_frames*3N)) sum_i
 * d/dtheta [ D_{v_i} y(x_i; theta) ] where D_v y is the directional derivative
 * of the MLP output along v (forward-mode tangent), differentiated in reverse
 * through both the primal and the tangent chain. */

static void o_descriptor_jvp(const o_system *sys, const o_potential *pot, int i, const o_nb *nb, int n,
                             const double *r, double *v) {
    int ns = sys->n_species, nr = pot->n_rbf, na = pot->n_ang;
    int d0 = o_input_dim(ns, nr, na);
    for (int f = 0; f < d0; ++f) v[f] = 0.0;
    for (int p = 0; p < n; ++p) {
        int sj = sys->species[nb[p].j];
        double rel = 0.0;   /* d-hat . (r_j - r_i) */
        for (int a = 0; a < 3; ++a) rel += nb[p].d[a] / nb[p].r * (r[3 * nb[p].j + a] - r[3 * i + a]);
        for (int k = 0; k < nr; ++k) {
            double g, dg;
            o_rbf(k, nr, pot->desc_cutoff, nb[p].r, &g, &dg);
            v[sj * nr + k] += dg * rel;
        }
    }
    for (int p = 0; p < n; ++p)
        for (int q2 = p + 1; q2 < n; ++q2)
            for (int a = 0; a < na; ++a) {
                double gp[3], gq[3];
                o_ang_term(a, pot->desc_cutoff, &nb[p], &nb[q2], gp, gq);
                double s = 0.0;
                for (int x3 = 0; x3 < 3; ++x3)
                    s += gp[x3] * (r[3 * nb[p].j + x3] - r[3 * i + x3]) + gq[x3] * (r[3 * nb[q2].j + x3] - r[3 * i + x3]);
                v[ns * nr + a] += s;
            }
}

/* Adds d(D_v y)/dtheta * scale into grad (packed like the weights). */
static void o_rop_grad(const o_potential *pot, int d0, const double *x, const double *v, double scale, double *grad) {
    o_layer L[16];
    const double *wout, *bout;
    o_layers(pot, d0, L, &wout, &bout);
    int W = pot->width, nl = pot->n_layers;
    double *h = (double *)malloc(sizeof(double) * (size_t)nl * W);
    double *hd = (double *)malloc(sizeof(double) * (size_t)nl * W);   /* tangent of h */
    double *a = (double *)malloc(sizeof(double) * (size_t)nl * W);
    double *ad = (double *)malloc(sizeof(double) * (size_t)nl * W);   /* tangent of a */
    /* forward primal + tangent */
    for (int l = 0; l < nl; ++l) {
        const double *in = l == 0 ? x : a + (size_t)(l - 1) * W;
        const double *ind = l == 0 ? v : ad + (size_t)(l - 1) * W;
        for (int o = 0; o < W; ++o) {
            double acc = L[l].b[o], accd = 0.0;
            for (int k = 0; k < L[l].din; ++k) {
                acc += L[l].W[(size_t)o * L[l].din + k] * in[k];
                accd += L[l].W[(size_t)o * L[l].din + k] * ind[k];
            }
            h[(size_t)l * W + o] = acc;
            hd[(size_t)l * W + o] = accd;
            a[(size_t)l * W + o] = o_silu(acc);
            ad[(size_t)l * W + o] = o_dsilu(acc) * accd;
        }
    }
    /* reverse: adjoints of a (primal) and ad (tangent); output yd = w_out . ad_L */
    double *ga = (double *)calloc((size_t)W, sizeof(double));
    double *gad = (double *)malloc(sizeof(double) * (size_t)W);
    double *gh = (double *)malloc(sizeof(double) * (size_t)W);
    double *ghd = (double *)malloc(sizeof(double) * (size_t)W);
    int dmax = W > d0 ? W : d0;
    double *ga_prev = (double *)malloc(sizeof(double) * (size_t)dmax);
    double *gad_prev = (double *)malloc(sizeof(double) * (size_t)dmax);
    /* packed offsets */
    int64_t *offW = (int64_t *)malloc(sizeof(int64_t) * (size_t)nl);
    int64_t *offb = (int64_t *)malloc(sizeof(int64_t) * (size_t)nl);
    int64_t off = 0;
    for (int l = 0; l < nl; ++l) { offW[l] = off; off += (int64_t)W * L[l].din; offb[l] = off; off += W; }
    int64_t offwout = off;
    for (int o = 0; o < W; ++o) {
        grad[offwout + o] += scale * ad[(size_t)(nl - 1) * W + o];   /* d yd / d w_out */
        gad[o] = wout[o];
        ga[o] = 0.0;
    }
    for (int l = nl - 1; l >= 0; --l) {
        for (int o = 0; o < W; ++o) {
            double hh = h[(size_t)l * W + o];
            ghd[o] = o_dsilu(hh) * gad[o];
            gh[o] = o_dsilu(hh) * ga[o] + o_d2silu(hh) * hd[(size_t)l * W + o] * gad[o];
        }
        const double *in = l == 0 ? x : a + (size_t)(l - 1) * W;
        const double *ind = l == 0 ? v : ad + (size_t)(l - 1) * W;
        int din = L[l].din;
        for (int o = 0; o < W; ++o) {
            grad[offb[l] + o] += scale * gh[o];
            for (int k = 0; k < din; ++k)
                grad[offW[l] + (int64_t)o * din + k] += scale * (gh[o] * in[k] + ghd[o] * ind[k]);
        }
        if (l > 0) {
            for (int k = 0; k < din; ++k) {
                double s1 = 0.0, s2 = 0.0;
                for (int o = 0; o < W; ++o) {
                    s1 += L[l].W[(size_t)o * din + k] * gh[o];
                    s2 += L[l].W[(size_t)o * din + k] * ghd[o];
                }
                ga_prev[k] = s1;
                gad_prev[k] = s2;
            }
            for (int k = 0; k < W; ++k) { ga[k] = ga_prev[k]; gad[k] = gad_prev[k]; }
        }
    }
    free(h); free(hd); free(a); free(ad); free(ga); free(gad); free(gh); free(ghd); free(ga_prev); free(gad_prev);
    free(offW); free(offb);
}

/* Returns the loss; grad (may be NULL) receives dL/dtheta for all packed
 * weights (b_out's entry is zero).  frames_q, frames_F: [n_frames][3N]. */
double o_force_match(const o_system *sys, const o_potential *draft, int32_t n_frames, const double *frames_q,
                     const double *frames_F, double *grad) {
    int N = sys->n_atoms, D = 3 * N, ns = sys->n_species;
    int d0 = o_input_dim(ns, draft->n_rbf, draft->n_ang);
    int64_t nw = o_n_weights(d0, draft->n_layers, draft->width);
    if (grad) for (int64_t k = 0; k < nw; ++k) grad[k] = 0.0;
    double *F = (double *)malloc(sizeof(double) * (size_t)D);
    double *r = (double *)malloc(sizeof(double) * (size_t)D);
    double *x = (double *)malloc(sizeof(double) * (size_t)d0);
    double *v = (double *)malloc(sizeof(double) * (size_t)d0);
    o_fix *fx = (o_fix *)malloc(sizeof(o_fix) * (size_t)N);
    o_nb *nb = (o_nb *)malloc(sizeof(o_nb) * O_NB_CAP);
    double loss = 0.0;
    double norm = 1.0 / ((double)n_frames * (double)D);
    for (int f = 0; f < n_frames; ++f) {
        const double *q = frames_q + (size_t)f * D;
        double E = o_energy_forces(sys, draft, q, F, NULL, NULL, NULL);
        if (isnan(E)) { loss = NAN; break; }
        for (int k = 0; k < D; ++k) {
            r[k] = F[k] - frames_F[(size_t)f * D + k];
            loss += norm * r[k] * r[k];
        }
        if (!grad) continue;
        o_fixpoint(sys, q, fx);
        for (int i = 0; i < N; ++i) {
            int n = o_list(sys, q, fx, i, draft->desc_cutoff, nb, O_NB_CAP);
            o_descriptor(sys, draft, i, nb, n, x);
            o_descriptor_jvp(sys, draft, i, nb, n, r, v);
            o_rop_grad(draft, d0, x, v, -2.0 * norm, grad);
        }
    }
    free(F); free(r); free(x); free(v); free(fx); free(nb);
    return loss;
}
