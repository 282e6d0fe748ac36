// Host build of the fixed-point sums of csrc/fixsum.cuh (the same source the step
// kernels compile), for the CPU tests: evaluates them on caller arrays.
#include "../../paper_2107_06355_gb300/csrc/fixsum.cuh"

using namespace pplbm::fx;

extern "C" {

// n nodes: f (n x 9 populations) -> out (n x 6): rho, jx, jy, m7, m8, valid (1 if the
// nine are in the range of the fixed-point path)
void fx_density(long long n, const double* f, double* out) {
  for (long long i = 0; i < n; ++i) {
    double v[9];
    for (int k = 0; k < 9; ++k) v[k] = f[9 * i + k];
    unsigned mx = 0;
    const bool ok = positive_normal_range(v, &mx);
    double* o = out + 6 * i;
    o[0] = o[1] = o[2] = o[3] = o[4] = 0.0;
    o[5] = ok ? 1.0 : 0.0;
    if (ok) density_moments<true>(v, frame_top(mx), &o[0], &o[1], &o[2], &o[3], &o[4]);
  }
}

// n nodes: p (n x 8: pE, pW, pN, pS, pNE, pNW, pSW, pSE) -> out (n x 2): gx, gy
void fx_stencil(long long n, const double* p, double* out) {
  for (long long i = 0; i < n; ++i) {
    const double* q = p + 8 * i;
    shan_chen_stencil(q[0], q[1], q[2], q[3], q[4], q[5], q[6], q[7], &out[2 * i], &out[2 * i + 1]);
  }
}
}

extern "C" {

// n rows of (j, h) -> out (n x 4): j + h, j + 2h, j + 3h, j - h
void fx_j_h(long long n, const double* in, double* out) {
  for (long long i = 0; i < n; ++i)
    j_h_combos<true>(in[2 * i], in[2 * i + 1], &out[4 * i], &out[4 * i + 1], &out[4 * i + 2], &out[4 * i + 3]);
}

// n rows of (r, xx, yy, xy, px, py, zz, p7, p8) -> out (n x 9) populations; shear != 0
// takes p7, p8 into account
void fx_populations(long long n, int shear, const double* in, double* out) {
  for (long long i = 0; i < n; ++i) {
    const double* q = in + 9 * i;
    double f[9];
    if (shear)
      reduced_populations<true>(q[0], q[1], q[2], q[3], q[4], q[5], q[6], q[7], q[8], f);
    else
      reduced_populations<false>(q[0], q[1], q[2], q[3], q[4], q[5], q[6], 0.0, 0.0, f);
    for (int k = 0; k < 9; ++k) out[9 * i + k] = f[k];
  }
}
}

extern "C" {

// n rows of mu (9) -> out (n x 9): the adjoints of reduced_populations' inputs
void fx_populations_transpose(long long n, int shear, const double* mu, double* out) {
  for (long long i = 0; i < n; ++i) {
    double m[9], o[9];
    for (int k = 0; k < 9; ++k) m[k] = mu[9 * i + k];
    if (shear)
      reduced_populations_transpose<true>(m, o);
    else
      reduced_populations_transpose<false>(m, o);
    for (int k = 0; k < 9; ++k) out[9 * i + k] = o[k];
  }
}

// n rows of (a1, a2, a3, a4, j0, h0) -> out (n x 2): jb, hb (with the j - h adjoint a4)
void fx_j_h_transpose(long long n, const double* in, double* out) {
  for (long long i = 0; i < n; ++i) {
    const double* q = in + 6 * i;
    j_h_combos_transpose<true>(q[0], q[1], q[2], q[3], q[4], q[5], &out[2 * i], &out[2 * i + 1]);
  }
}
}

extern "C" {

// n rows of 13 gather inputs -> out (n): psi_adjoint_gather
void fx_psi_gather(long long n, const double* in, double* out) {
  for (long long i = 0; i < n; ++i) {
    double v[13];
    for (int k = 0; k < 13; ++k) v[k] = in[13 * i + k];
    out[i] = psi_adjoint_gather(v);
  }
}

// n rows of (rho_b, jx_b, jy_b, m7_b, m8_b) -> out (n x 9): lambda_assembly
void fx_lambda(long long n, int shear, const double* in, double* out) {
  for (long long i = 0; i < n; ++i) {
    const double* q = in + 5 * i;
    double l[9];
    if (shear)
      lambda_assembly<true>(q[0], q[1], q[2], q[3], q[4], l);
    else
      lambda_assembly<false>(q[0], q[1], q[2], q[3], q[4], l);
    for (int k = 0; k < 9; ++k) out[9 * i + k] = l[k];
  }
}
}
