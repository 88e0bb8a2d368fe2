// Internal declarations of the GB300 PUFE library: the context, error
// helpers and the basis functions shared by the host setup and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/pufe.h"

namespace pufe {

// ---------------------------------------------------------------------------
// error reporting
// ---------------------------------------------------------------------------
void set_error(const std::string &msg);
pufe_status fail(pufe_status st, const std::string &msg);
pufe_status cuda_fail(cudaError_t err, const char *what);

#define PUFE_CUDA_TRY(call)                                   \
  do {                                                        \
    cudaError_t _e = (call);                                  \
    if (_e != cudaSuccess) return ::pufe::cuda_fail(_e, #call); \
  } while (0)

// device-side error flag bits
enum : unsigned {
  DEVERR_BOUNDS = 1u,   // an index check failed inside a kernel
  DEVERR_TIMEOUT = 2u,  // a bounded wait gave up
  DEVERR_SHAPE = 4u,    // a kernel met a shape it was not built for
  DEVERR_NONFINITE = 8u // an input (V) held a NaN or an infinity
};

// ---------------------------------------------------------------------------
// one enrichment function alpha = (atom, orbital)
// ---------------------------------------------------------------------------
struct Orbital {
  double tau[3];   // atom position
  double zeta;     // Slater exponent
  double norm;     // STO normalisation (2 zeta)^(n+1/2) / sqrt((2n)!)
  double rc;       // cutoff radius
  int n, l, m;
  int pad;
};

// the same enrichment with FP32 parameters (mixed-precision path)
struct OrbitalF {
  float zeta, norm, rc, inv_rc;
  int n, l, m, pad;
};

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
struct ProjDev;

struct DeviceArrays {
  // quadrature
  int64_t *qoff = nullptr;    // nelem + 1
  double *x = nullptr;        // nq * 3
  double *w = nullptr;        // nq
  double *xi = nullptr;       // nq * 3, reference coordinates in [-1, 1]
  // element basis description
  int64_t *doff = nullptr;    // nelem + 1: offsets into dofs (n_e each)
  int32_t *dofs = nullptr;    // sum n_e: global DOF of each element column
  int32_t *ecol = nullptr;    // sum (n_e - 64): (aslot << 3) | local vertex
  uint8_t *eshift = nullptr;  // sum n_e: lattice shift bits of each column (Bloch phases)
  int32_t *aoff = nullptr;    // nelem + 1: offsets into alist
  int32_t *alist = nullptr;   // element enrichment list (global alpha ids)
  int64_t *toff = nullptr;    // nelem + 1: offsets into psi (units of q*alpha)
  double *psi = nullptr;      // 4 * sum Q_e A_e: [aslot][comp][q] per element
  // FP32 (mixed-precision) path: element points padded to a multiple of 8
  int64_t *qpoff = nullptr;   // nelem + 1: offsets into qdat (padded points)
  float4 *qdat = nullptr;     // per padded point: (xi_x, xi_y, xi_z, w); w = 0 on padding
  float *ptab = nullptr;      // per padded point, 32 floats: L[3][4], dL[3][4] (x 2/h),
                              // xi[3], sqrt(w/2), sqrt(w), 3 unused; zeros on padding
  float *vpad = nullptr;      // per padded point: FP32 copy of V (filled per call)
  // tensor structure of the rules: per element a list of (sub)cells, each a
  // p^3 Gauss rule whose points are consecutive (x fastest)
  int32_t *partoff = nullptr; // nelem + 1: offsets into part arrays
  int32_t *part_p = nullptr;  // points per axis of each part
  int32_t *part_q = nullptr;  // first point of each part (relative to the element)
  int64_t *toff32 = nullptr;  // nelem + 1: offsets into psi32 (units of padded q*alpha)
  float *psi32 = nullptr;     // per element [q/8][slot][comp][q%8]: 32-float blocks
  float *eorig = nullptr;     // per (element, slot): displacement of the element
                              // origin from the nearest atom image, hi[3], lo[3], 0, 0
  double *Tfe = nullptr;      // 64 x 64: kinetic block of the tricubic functions (any element)
  double *Sfe = nullptr;      // 64 x 64: overlap block of the tricubic functions (any element)
  double *S0 = nullptr;       // nnz: overlap FE-FE constants summed over elements (mixed path)
  Orbital *orb = nullptr;     // n_alpha
  OrbitalF *orbf = nullptr;   // n_alpha
  // global sparse storage
  int64_t *rowptr = nullptr;  // N + 1
  int32_t *col = nullptr;     // nnz
  int64_t *soff = nullptr;    // nelem + 1: offsets into smap (n_e^2 each)
  int32_t *smap = nullptr;    // CSR slot of each local pair (i, j), row-major
  // work list: elements sorted by (n_e, Q_e) class, largest first
  int32_t *order = nullptr;   // nelem
  // FP64 assembly/adjoint work list, 3 per item (element, first point, end
  // point), largest first; null when every item is a whole element
  int32_t *wsplit = nullptr;
  // mixed-path work list of the n_e > 128 elements, 3 per item (index into
  // `order`, first chunk, end chunk; chunks of 8 padded points), largest first
  int32_t *titems = nullptr;
  int32_t *sitems = nullptr;   // E-E kernel of S: (order index, first pair, end pair) triples
  // E-E block of S in the Gram form, 5 per item: (order index, row tile,
  // column tile, first point, end point); tiles of 32 (gitems32) or 64 columns
  int32_t *gitems32 = nullptr, *gitems64 = nullptr;
  int32_t *citems = nullptr;   // strip kernel: (order index, first cell, end cell) triples
  int32_t *pitems = nullptr;   // FP32 density / per-point adjoint: (order index, first point, end point)
  int32_t *tblk = nullptr;     // nelem + 1: FP32 tabulation CTAs per element, prefix summed
  int8_t *eeform = nullptr;   // per element: E x E form of the strip (0 model, 1 pair, 2 direct)
  unsigned *err = nullptr;    // device error flag
  // side stream and events: the FE-FE kernel of the mixed assembly runs on
  // `side`, forked from and joined back into the caller's stream
  cudaStream_t side = nullptr;
  ProjDev *proj = nullptr;     // 64 projector descriptions (allocated on first use)
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
};

}  // namespace pufe

namespace pufe {
struct ScfState;
}

struct pufe_ctx {
  int device = 0;
  double a[3] = {0, 0, 0};
  double h[3] = {0, 0, 0};
  bool general = false;        // a general (triclinic) cell: lat, Jit below
  bool ser = false;            // FE space: cubic serendipity (32 columns) instead of tricubic
  int nfe_e = 64;              // FE columns per element (64 tricubic, 32 serendipity)
  double lat[9] = {0};         // rows a_1, a_2, a_3 (general cells)
  double Jit[9] = {0};         // J^-T (general cells): physical gradient = Jit grad_xi
  int nel[3] = {0, 0, 0};
  int images[3] = {1, 1, 1};   // image search half-width per axis
  int64_t nelem = 0, nq = 0, n_dof = 0, n_fe = 0, nnz = 0;
  int64_t n_alpha = 0, psi_len = 0, smap_len = 0, dof_len = 0;
  int64_t nq_pad = 0, psi32_len = 0;
  int max_basis = 0, max_q = 0, max_alpha = 0;
  bool tabulated = false;     // FP64 enrichment table is current
  bool tabulated32 = false;   // FP32 enrichment table is current
  bool fe_exact = false;      // every rule has >= 4 points per axis per (sub)cell
  int n_big = 0;              // elements with n_e > 128 (listed first in `order`)
  int64_t big_pad_end = 0;    // end of the last n_e > 128 element's padded points (0: none)
  int64_t n_wsplit = 0;       // items of the FP64 point-range work list (0: none)
  int n_titems = 0;           // items of the mixed path's list for the n_e > 128 elements
  int n_sitems = 0;           // items of the E-E overlap kernel's list (slot-pair ranges)
  int n_gitems32 = 0, n_gitems64 = 0;   // items of the Gram-form lists
  int n_citems = 0;           // items of the strip kernel's list ((sub)cell ranges)
  int n_pitems = 0;           // items of the FP32 per-point list (point ranges of every element)
  int n_tblk = 0;             // CTAs of the FP32 tabulation (TAB_CHUNK table items each)
  int max_part_p = 0;         // largest points-per-axis of any (sub)cell
  int strip_stage = 0;        // floats of the strip kernel's shared-memory stage
  uint32_t strip_pmask = 0;   // per-axis counts (bit p) of the strip kernel's cells
  int strip_npair_max = 0;    // most enrichment pairs A (A + 1) / 2 of a strip element, A <= 8
  int adj_sf_floats = 0;      // shared floats of the slot-form adjoint strip's coefficients and Psi
  bool adj_sf_all = true;     // every strip element takes the slot-form adjoint
  bool on_device = false;   // device copies exist (a CUDA device was present)
  // host copies kept for getters
  std::vector<int64_t> qoff, rowptr, doff;
  std::vector<int32_t> col, dofs, n_e, q_e, order;
  std::vector<int32_t> see_stage;   // per element: slots x largest (sub)cell's points (0: no strip)
  std::vector<int32_t> n_slot;      // per element: enrichments (slots) in its basis
  std::vector<std::vector<int32_t>> part_p_host;   // per element: points per axis of each (sub)cell
  std::vector<int8_t> eeform_host;  // per element: E x E form (0 model, 1 pair, 2 direct)
  // instrumentation of the mixed assembly (pufe_profile_assembly): events
  // around the call [0, 1], the FE-FE kernel [2, 3], the FP64 E-E kernel of
  // S [4, 5], the tensor-core tile [6, 7] and the strip [8, 9]
  bool prof = false;
  bool prof_ran[5] = {false, false, false, false, false};
  cudaEvent_t pev[10] = {nullptr, nullptr, nullptr, nullptr, nullptr,
                         nullptr, nullptr, nullptr, nullptr, nullptr};
  std::vector<double> x, w;
  pufe::DeviceArrays d;
  pufe::ScfState *scf = nullptr;   // SCF work arrays, made on first use
};

namespace pufe {

// Elements (n_e <= 128) whose enrichment strip of the adjoint runs in the
// slot form: at most 16 enrichment slots and 10 points per axis per (sub)cell.
__host__ __device__ inline bool adjoint_sf_fits(int A, int pmax) { return A <= 16 && pmax <= 10; }
// (slot, padded point) items of the FP32 enrichment table per tabulation CTA
constexpr int TAB_CHUNK = 2048;
// Shared-memory stage of the E-E overlap kernel (floats): elements whose
// slots' Psi values on one (sub)cell exceed it take the Gram form instead
constexpr int SEE_STAGE_MAX_F = 8192;
// points per Gram-form work item
constexpr int GRAM_QCHUNK = 128;

// ---------------------------------------------------------------------------
// basis functions shared by host setup and device kernels
// ---------------------------------------------------------------------------

// Cubic Lagrange polynomials on nodes -1, -1/3, 1/3, 1 and their slopes.
__host__ __device__ inline void lagrange3(double t, double L[4], double dL[4]) {
  const double a = t + 1.0, b = t + 1.0 / 3.0, c = t - 1.0 / 3.0, d = t - 1.0;
  L[0] = -0.5625 * b * c * d;
  L[1] = 1.6875 * a * c * d;
  L[2] = -1.6875 * a * b * d;
  L[3] = 0.5625 * a * b * c;
  dL[0] = -0.5625 * (c * d + b * d + b * c);
  dL[1] = 1.6875 * (c * d + a * d + a * c);
  dL[2] = -1.6875 * (b * d + a * d + a * b);
  dL[3] = 0.5625 * (b * c + a * c + a * b);
}

// Cubic serendipity hexahedron (32 nodes; the classical FE part of the
// paper's PUFE runs, Sec. 6): its nodes are the tricubic nodes with at most
// one index inner (the 8 vertices and two inner nodes per edge).  Column c
// (0..31) is the local tricubic node ser_local(c) = a + 4 b + 16 c, in
// ascending order.
__host__ __device__ inline int ser_local(int c) {
  constexpr unsigned char t[32] = {0,  1,  2,  3,  4,  7,  8,  11, 12, 13, 14,
                                   15, 16, 19, 28, 31, 32, 35, 44, 47, 48, 49,
                                   50, 51, 52, 55, 56, 59, 60, 61, 62, 63};
  return t[c];
}

// Value and reference gradient of serendipity column c at xi:
//   vertex s in {-1, 1}^3:  N = 1/64 prod_d (1 + s_d xi_d) (9 |xi|^2 - 19);
//   inner node of an edge along axis d (coordinate t = -+1/3, the others
//   s_e = -+1):  N = 9/64 (1 - xi_d^2) (1 + 9 t xi_d) prod_{e != d} (1 + s_e xi_e).
__host__ __device__ inline void serendipity32(int c, const double xi[3], double &N, double g[3]) {
  const int loc = ser_local(c);
  const int idx[3] = {loc & 3, (loc >> 2) & 3, loc >> 4};
  double nd[3];
  int inner = -1;
  for (int d = 0; d < 3; ++d) {
    nd[d] = idx[d] == 0 ? -1.0 : (idx[d] == 1 ? -1.0 / 3.0 : (idx[d] == 2 ? 1.0 / 3.0 : 1.0));
    if (idx[d] == 1 || idx[d] == 2) inner = d;
  }
  if (inner < 0) {
    const double l0 = 1.0 + nd[0] * xi[0], l1 = 1.0 + nd[1] * xi[1], l2 = 1.0 + nd[2] * xi[2];
    const double G = 9.0 * (xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2]) - 19.0;
    const double P = l0 * l1 * l2;
    N = P * G / 64.0;
    g[0] = (nd[0] * l1 * l2 * G + P * 18.0 * xi[0]) / 64.0;
    g[1] = (nd[1] * l0 * l2 * G + P * 18.0 * xi[1]) / 64.0;
    g[2] = (nd[2] * l0 * l1 * G + P * 18.0 * xi[2]) / 64.0;
    return;
  }
  const int d = inner, e1 = (d + 1) % 3, e2 = (d + 2) % 3;
  const double t = nd[d], x = xi[d];
  const double f = (1.0 - x * x) * (1.0 + 9.0 * t * x);
  const double fp = -2.0 * x * (1.0 + 9.0 * t * x) + 9.0 * t * (1.0 - x * x);
  const double l1 = 1.0 + nd[e1] * xi[e1], l2 = 1.0 + nd[e2] * xi[e2];
  N = 9.0 / 64.0 * f * l1 * l2;
  g[d] = 9.0 / 64.0 * fp * l1 * l2;
  g[e1] = 9.0 / 64.0 * f * nd[e1] * l2;
  g[e2] = 9.0 / 64.0 * f * l1 * nd[e2];
}

// Real solid harmonic r^l Y_lm(r^) (unit-normalised Y, no Condon-Shortley
// phase, m < 0 <-> sin) and its gradient, for l <= 3.  T = double or float.
template <class T>
__host__ __device__ inline T solid_harmonic(int l, int m, T x, T y, T z, T g[3]) {
  const T PI = T(3.14159265358979323846);
  g[0] = g[1] = g[2] = T(0);
  if (l == 0) return T(0.28209479177387814);  // 1 / (2 sqrt(pi))
  if (l == 1) {
    const T c = T(0.48860251190291992);       // sqrt(3 / (4 pi))
    if (m == -1) { g[1] = c; return c * y; }
    if (m == 0) { g[2] = c; return c * z; }
    g[0] = c; return c * x;
  }
  if (l == 2) {
    const T A = T(1.0925484305920792);        // sqrt(15/pi) / 2
    const T B = T(0.31539156525252005);       // sqrt(5/pi) / 4
    const T C = T(0.54627421529603959);       // sqrt(15/pi) / 4
    switch (m) {
      case -2: g[0] = A * y; g[1] = A * x; return A * x * y;
      case -1: g[1] = A * z; g[2] = A * y; return A * y * z;
      case 0: g[0] = -2 * B * x; g[1] = -2 * B * y; g[2] = 4 * B * z;
        return B * (2 * z * z - x * x - y * y);
      case 1: g[0] = A * z; g[2] = A * x; return A * x * z;
      default: g[0] = 2 * C * x; g[1] = -2 * C * y; return C * (x * x - y * y);
    }
  }
  (void)PI;
  const T D = T(0.59004358992664352);         // sqrt(35/(2 pi)) / 4
  const T E = T(2.8906114426405538);          // sqrt(105/pi) / 2
  const T F = T(0.45704579946446572);         // sqrt(21/(2 pi)) / 4
  const T G = T(0.37317633259011540);         // sqrt(7/pi) / 4
  const T H = T(1.4453057213202769);          // sqrt(105/pi) / 4
  switch (m) {
    case -3: g[0] = 6 * D * x * y; g[1] = 3 * D * (x * x - y * y); return D * y * (3 * x * x - y * y);
    case -2: g[0] = E * y * z; g[1] = E * x * z; g[2] = E * x * y; return E * x * y * z;
    case -1: g[0] = -2 * F * x * y; g[1] = F * (4 * z * z - x * x - 3 * y * y); g[2] = 8 * F * y * z;
      return F * y * (4 * z * z - x * x - y * y);
    case 0: g[0] = -6 * G * x * z; g[1] = -6 * G * y * z; g[2] = G * (6 * z * z - 3 * x * x - 3 * y * y);
      return G * z * (2 * z * z - 3 * x * x - 3 * y * y);
    case 1: g[0] = F * (4 * z * z - 3 * x * x - y * y); g[1] = -2 * F * x * y; g[2] = 8 * F * x * z;
      return F * x * (4 * z * z - x * x - y * y);
    case 2: g[0] = 2 * H * x * z; g[1] = -2 * H * y * z; g[2] = H * (x * x - y * y);
      return H * z * (x * x - y * y);
    default: g[0] = 3 * D * (x * x - y * y); g[1] = -6 * D * x * y; return D * x * (x * x - 3 * y * y);
  }
}

template <class T>
__host__ __device__ inline T ipow(T r, int k) {
  T p = T(1);
  for (int i = 0; i < k; ++i) p *= r;
  return p;
}

// Psi~(d) h(|d|, r_c) for one image displacement d, plus its gradient
// (accumulated into psi and g).  Psi~ = N r^(n-1) e^(-zeta r) Y_lm, written
// as f(r) S_lm(d) with f = N r^(n-1-l) e^(-zeta r) h(r) and S_lm = r^l Y_lm.
template <class T>
__host__ __device__ inline void orbital_accumulate(const Orbital &o, T dx, T dy, T dz, T &psi,
                                                   T g[3]) {
  const T rc = T(o.rc);
  const T r2 = dx * dx + dy * dy + dz * dz;
  if (r2 >= rc * rc) return;
  const T r = sqrt(r2);
  const T x = r / rc;
  const T x3 = x * x * x;
  const T hc = T(1) + x3 * x * (T(-35) + x * (T(84) + x * (T(-70) + T(20) * x)));
  const T omx = T(1) - x;
  const T dh = T(-140) * x3 * omx * omx * omx / rc;
  const int k = o.n - 1 - o.l;  // >= 0
  const T ez = T(o.norm) * exp(-T(o.zeta) * r);
  const T rk = ipow(r, k);
  const T f = ez * rk * hc;
  const T rkm1 = (k > 0) ? ipow(r, k - 1) : T(0);
  const T df = ez * (T(k) * rkm1 * hc - T(o.zeta) * rk * hc + rk * dh);
  T gs[3];
  const T S = solid_harmonic<T>(o.l, o.m, dx, dy, dz, gs);
  psi += f * S;
  if (r > T(1e-14)) {
    const T s = df * S / r;
    g[0] += s * dx + f * gs[0];
    g[1] += s * dy + f * gs[1];
    g[2] += s * dz + f * gs[2];
  } else {
    g[0] += f * gs[0];
    g[1] += f * gs[1];
    g[2] += f * gs[2];
  }
}

// A general (triclinic) cell for the image sums: rows a_d of the lattice
// (L[3 d + c]), L^-T (Lit), and the image half-width per lattice direction.
struct LatticeDev {
  double L[9], Lit[9];
  int img[3];
};

// Periodic enrichment Psi_alpha(p) of a general cell: the displacement to the
// atom is rounded in lattice coordinates, s = L^-T d, s <- s - nearest
// integer, d_0 = L^T s, then every image d_0 + i a_1 + j a_2 + k a_3 within
// the image half-widths is summed (terms beyond r_c are zero).
template <class T>
__host__ __device__ inline void enrichment_eval_lat(const Orbital &o, const double p[3],
                                                    const LatticeDev &c, T &psi, T g[3]) {
  psi = T(0);
  g[0] = g[1] = g[2] = T(0);
  double d[3], s[3];
  for (int k = 0; k < 3; ++k) d[k] = p[k] - o.tau[k];
  for (int k = 0; k < 3; ++k) {
    s[k] = c.Lit[3 * k] * d[0] + c.Lit[3 * k + 1] * d[1] + c.Lit[3 * k + 2] * d[2];
    s[k] -= floor(s[k] + 0.5);
  }
  double d0[3];
  for (int k = 0; k < 3; ++k) d0[k] = s[0] * c.L[k] + s[1] * c.L[3 + k] + s[2] * c.L[6 + k];
  for (int i = -c.img[0]; i <= c.img[0]; ++i)
    for (int j = -c.img[1]; j <= c.img[1]; ++j)
      for (int k = -c.img[2]; k <= c.img[2]; ++k) {
        double r[3];
        for (int m = 0; m < 3; ++m) r[m] = d0[m] + i * c.L[m] + j * c.L[3 + m] + k * c.L[6 + m];
        orbital_accumulate<T>(o, T(r[0]), T(r[1]), T(r[2]), psi, g);
      }
}

// Periodic enrichment Psi_alpha(p) (eq. Psi with f(R) = 1): all images of the
// atom within r_c of p.  `img` = image half-width per axis.  The displacement
// to the nearest image is formed in double precision, then evaluated in T.
template <class T>
__host__ __device__ inline void enrichment_eval(const Orbital &o, const double p[3],
                                                const double a[3], const int img[3], T &psi,
                                                T g[3]) {
  psi = T(0);
  g[0] = g[1] = g[2] = T(0);
  double d0[3];
  for (int k = 0; k < 3; ++k) {
    double d = p[k] - o.tau[k];
    d -= a[k] * floor(d / a[k] + 0.5);
    d0[k] = d;
  }
  for (int i = -img[0]; i <= img[0]; ++i)
    for (int j = -img[1]; j <= img[1]; ++j)
      for (int k = -img[2]; k <= img[2]; ++k)
        orbital_accumulate<T>(o, T(d0[0] + i * a[0]), T(d0[1] + j * a[1]), T(d0[2] + k * a[2]),
                              psi, g);
}

// launchers implemented in the .cu files
pufe_status launch_tabulate(pufe_ctx *ctx, cudaStream_t s);
pufe_status launch_assemble_fp64(pufe_ctx *ctx, const double *V, int what, double *H, double *S,
                                 cudaStream_t s);
pufe_status launch_density_fp64(pufe_ctx *ctx, const double *C, int64_t ldc, const double *f,
                                int nocc, double *rho, cudaStream_t s);
pufe_status launch_adjoint_fp64(pufe_ctx *ctx, const double *Hbar, double *Vbar, cudaStream_t s);
// Gaussian nonlocal projector on the device: N r^l exp(-r^2/(2 rp^2)) Y_lm,
// images within rcut
struct ProjDev {
  double tau[3];
  double rp, N, rcut;
  int l, m;
};
// k == nullptr: Gamma point, F real; else F + i Fi at wavevector k
pufe_status launch_projections(pufe_ctx *ctx, const ProjDev *pj, int P, const double *k, double *F,
                               double *Fi, cudaStream_t s);
// Bloch (k != 0) FP64 variants: phases exp(i k . R) of the 8 shift codes
struct PhaseTab {
  double re[8], im[8];
};
PhaseTab phase_table(const pufe_ctx *ctx, const double k[3]);
// Cotangent of the FP32 adjoint kernels at a wavevector: the complex
// Hbar + i Hi enters through the real element block
// Re(conj(Hbar + i Hi)[g_i, g_j] exp(i k.(R_j - R_i))) (the derivative of
// Re sum conj(Hbar) H(k)); Hi == nullptr is the Gamma point, Hbar real.
struct BlochCot {
  const double *Hi;
  const uint8_t *eshift;   // shift code of every element column (sum n_e)
  PhaseTab ph;
};
// entry of that block from the two CSR values and the columns' shift codes
__host__ __device__ inline double cot_entry(double hr, double hi, int ci, int cj,
                                            const PhaseTab &ph) {
  if (ci == cj) return hr;
  const double pr = ph.re[ci] * ph.re[cj] + ph.im[ci] * ph.im[cj];
  const double pim = ph.re[ci] * ph.im[cj] - ph.im[ci] * ph.re[cj];
  return hr * pr + hi * pim;
}
pufe_status launch_assemble_fp64_bloch(pufe_ctx *ctx, const PhaseTab &ph, const double *V,
                                       int what, double *H, double *Hi, double *S, double *Si,
                                       cudaStream_t s);
pufe_status launch_density_fp64_bloch(pufe_ctx *ctx, const PhaseTab &ph, const double *Cr,
                                      const double *Ci, int64_t ldc, const double *f, int nocc,
                                      double *rho, cudaStream_t s);
pufe_status launch_adjoint_fp64_bloch(pufe_ctx *ctx, const PhaseTab &ph, const double *Hr,
                                      const double *Hi, double *Vbar, cudaStream_t s);
pufe_status launch_tabulate_f32(pufe_ctx *ctx, cudaStream_t s);
// FP32 adjoint; bc != nullptr: at a wavevector (complex cotangent)
pufe_status launch_adjoint_tc(pufe_ctx *ctx, const double *Hbar, double *Vbar, cudaStream_t s,
                              const BlochCot *bc = nullptr);
// adds the FE-FE blocks of H (kinetic constants + V term; V == NULL: V = 0)
pufe_status launch_fefe(pufe_ctx *ctx, const double *V, double *H, cudaStream_t s);
pufe_status launch_strip_sf(pufe_ctx *ctx, const double *V, int what, double *H, double *S,
                            int first, int count, cudaStream_t s);
pufe_status launch_fefe_bloch(pufe_ctx *ctx, const PhaseTab &ph, const double *V, int what,
                              double *H, double *Hi, double *S, double *Si, cudaStream_t s);
// mixed-precision Bloch assembly (n_e <= 128): FE-FE blocks with FP64 phases,
// the enrichment strip in FP32 with FP32 phases; outputs zeroed here
pufe_status launch_assemble_mixed_bloch(pufe_ctx *ctx, const PhaseTab &ph, const double *V,
                                        int what, double *H, double *Hi, double *S, double *Si,
                                        cudaStream_t s);
pufe_status scf_prepare(pufe_ctx *ctx);
void scf_free(pufe_ctx *ctx);
pufe_status launch_ion_density(pufe_ctx *ctx, int natoms, const double *tau, const double *Z,
                               const double *sigma, double *rho, cudaStream_t s);
pufe_status launch_effective_potential(pufe_ctx *ctx, const double *n, const double *rho_I,
                                       double *V_eff, double *V_C, double *eps_xc, cudaStream_t s);
void scf_reset(pufe_ctx *ctx);
pufe_status launch_scf_step(pufe_ctx *ctx, int nstates, const double *eps, const double *C,
                            int64_t ldc, double nelec, double kT, double alpha, int pulay, int prec,
                            const double *rho_I, const double *V_eff_in, double *n, double *V_eff_out,
                            double *f_out, pufe_scf_info *info, cudaStream_t s);
pufe_status launch_scf_step_bloch(pufe_ctx *ctx, int nk, const double *kpts, const double *wk,
                                  int nstates, const double *eps, const double *const *C_re,
                                  const double *const *C_im, int64_t ldc, double nelec, double kT,
                                  double alpha, int pulay, int prec, const double *rho_I,
                                  const double *V_eff_in, double *n, double *V_eff_out,
                                  double *f_out, pufe_scf_info *info, cudaStream_t s);
pufe_status launch_adjoint_fefe(pufe_ctx *ctx, const double *Hbar, double *Vbar, int first,
                                int count, cudaStream_t s, const BlochCot &bc);
pufe_status launch_adjoint_strip_sf(pufe_ctx *ctx, const double *Hbar, double *Vbar, int first,
                                    int count, cudaStream_t s, const BlochCot &bc);
// S enrichment-enrichment block with FP64-class sums (mixed path): adds into S (and Si at
// a wavevector: ph != nullptr) for every element, over the slot-pair work list
pufe_status launch_see(pufe_ctx *ctx, const PhaseTab *ph, double *S, double *Si, cudaStream_t s);
// one bounded mbarrier wait that nothing completes (diagnostics of the
// timeout path): gives up after wait_ns and sets DEVERR_TIMEOUT
pufe_status launch_wait_probe(pufe_ctx *ctx, uint64_t wait_ns, cudaStream_t st);
// autotuner of the strip's E x E form per element class (blocking)
pufe_status autotune_strip(pufe_ctx *ctx, int *ntuned, cudaStream_t st);
// instrumentation of the mixed assembly (events around its kernels)
pufe_status profile_enable(pufe_ctx *ctx, bool on);
pufe_status profile_read(pufe_ctx *ctx, double ms[5]);
pufe_status launch_assemble_tc_static(pufe_ctx *ctx, const double *V, int what, double *H,
                                      double *S, cudaStream_t s);
pufe_status launch_assemble_tc(pufe_ctx *ctx, const double *V, int what, double *H, double *S,
                               cudaStream_t s);
// FP32 density; Ci != nullptr: Bloch states C + i Ci at the wavevector of ph
pufe_status launch_density_tc(pufe_ctx *ctx, const double *C, int64_t ldc, const double *f,
                              int nocc, double *rho, cudaStream_t s, const double *Ci = nullptr,
                              const PhaseTab *ph = nullptr);

}  // namespace pufe
