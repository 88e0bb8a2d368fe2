// Self-consistent-field step (Sec. 3): ionic charge, total Coulomb potential,
// LDA exchange-correlation, occupations, density mixing and total energy.
//
// Coulomb potential.  Sec. 3 (eq. poisson) obtains V_C = V_I + V_H from one
// Poisson equation for the total charge rho = rho_I - n (Gaussian ionic
// charges, electrons with density n).  It is solved in the tricubic FE space
// of the mesh:  -K v = 4 pi b,  K_ij = int grad phi_i . grad phi_j,
// b_i = int phi_i rho (shared element rule), zero cell average.  The mesh is
// a periodic tensor grid, so K = K1 (x) M1 (x) M1 + M1 (x) K1 (x) M1 +
// M1 (x) M1 (x) K1 with the 1D periodic cubic stiffness K1 and mass M1 of each
// axis.  With the 1D generalized eigenvectors X (K1 X = M1 X Lambda,
// X^T M1 X = I), K^+ = (X (x) X (x) X) D^+ (X (x) X (x) X)^T with
// D = Lambda_x + Lambda_y + Lambda_z: the solve is three small dense
// transforms along the axes, a diagonal scaling with the constant mode set to
// zero (which is exactly the zero-average solution), and three transforms
// back (the fast diagonalization method of Lynch, Rice and Thomas, 1964).
//
// LDA: Dirac exchange plus the Perdew-Zunger 1981 fit of the Ceperley-Alder
// correlation, unpolarised (the paper names the LDA without its fit).
// Everything here is FP64.
#include <algorithm>
#include <cmath>
#include <vector>

#include "pufe_internal.h"

namespace pufe {

// per-context work arrays of the SCF calls (allocated on first use)
struct ScfState {
  int n1[3] = {0, 0, 0};
  double *X[3] = {nullptr, nullptr, nullptr};     // n1 x n1, row-major X[node][mode]
  double *lam[3] = {nullptr, nullptr, nullptr};   // n1, ascending
  double *b = nullptr, *t0 = nullptr, *t1 = nullptr;   // n_fe each
  double *n_out = nullptr, *vc = nullptr, *exc = nullptr, *vxc = nullptr;   // n_q each
  double *sums = nullptr;   // 8 reduction slots
  double *f = nullptr;      // occupations: 64 states x up to 64 k-points (k-major)
  double *nk = nullptr;     // n_q: one k-point's density (k-point steps)
  double *atoms = nullptr;  // 5 per atom: tau (3), Z, sigma
  int atoms_cap = 0;
  double e_self = 0.0;      // self-energy of the last ionic charge set
  // Pulay history: ring of PULAY_MAX (input density, residual) pairs
  double *hist_n = nullptr, *hist_R = nullptr, *dots = nullptr;
  std::vector<int> slots;   // active slots, oldest first
  double gram[8][8] = {{0}};
  int next_slot = 0;
};

namespace {

constexpr double PI = 3.14159265358979323846;

// ---------------------------------------------------------------------------
// host: 1D periodic cubic FE matrices and their generalized eigenvectors
// ---------------------------------------------------------------------------

// cyclic Jacobi rotations: A (n x n, symmetric, row-major) -> Q Lambda Q^T
static void jacobi_eigen(int n, std::vector<double> &A, std::vector<double> &Q,
                         std::vector<double> &lam) {
  Q.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) Q[(size_t)i * n + i] = 1.0;
  double norm = 0.0;
  for (double v : A) norm += v * v;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = i + 1; j < n; ++j) off += A[(size_t)i * n + j] * A[(size_t)i * n + j];
    if (off <= 1e-32 * norm) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = A[(size_t)p * n + q];
        if (std::fabs(apq) < 1e-300) continue;
        const double app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
        const double theta = (aqq - app) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {   // A <- J^T A J, columns p and q
          const double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
          A[(size_t)k * n + p] = c * akp - s * akq;
          A[(size_t)k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {   // rows p and q
          const double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
          A[(size_t)p * n + k] = c * apk - s * aqk;
          A[(size_t)q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          const double qkp = Q[(size_t)k * n + p], qkq = Q[(size_t)k * n + q];
          Q[(size_t)k * n + p] = c * qkp - s * qkq;
          Q[(size_t)k * n + q] = s * qkp + c * qkq;
        }
      }
  }
  lam.resize(n);
  for (int i = 0; i < n; ++i) lam[i] = A[(size_t)i * n + i];
}

// K1 X = M1 X Lambda, X^T M1 X = I for the periodic 1D cubic space of nel
// elements of length h (3 nel nodes); modes sorted by ascending Lambda
static void axis_modes(int nel, double h, std::vector<double> &X, std::vector<double> &lam) {
  const int n = 3 * nel;
  // 4-point Gauss-Legendre (exact for the degree-6 mass integrand)
  const double a = std::sqrt(3.0 / 7.0 - 2.0 / 7.0 * std::sqrt(6.0 / 5.0));
  const double b = std::sqrt(3.0 / 7.0 + 2.0 / 7.0 * std::sqrt(6.0 / 5.0));
  const double wa = (18.0 + std::sqrt(30.0)) / 36.0, wb = (18.0 - std::sqrt(30.0)) / 36.0;
  const double gx[4] = {-b, -a, a, b}, gw[4] = {wb, wa, wa, wb};
  double Ke[4][4] = {{0}}, Me[4][4] = {{0}};
  for (int g = 0; g < 4; ++g) {
    double L[4], dL[4];
    lagrange3(gx[g], L, dL);
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) {
        Me[i][j] += gw[g] * L[i] * L[j] * (h / 2.0);
        Ke[i][j] += gw[g] * dL[i] * dL[j] * (2.0 / h);
      }
  }
  std::vector<double> K((size_t)n * n, 0.0), M((size_t)n * n, 0.0);
  for (int e = 0; e < nel; ++e)
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) {
        const int gi = (3 * e + i) % n, gj = (3 * e + j) % n;
        K[(size_t)gi * n + gj] += Ke[i][j];
        M[(size_t)gi * n + gj] += Me[i][j];
      }
  // M = L L^T
  std::vector<double> Lc((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j <= i; ++j) {
      double s = M[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) s -= Lc[(size_t)i * n + k] * Lc[(size_t)j * n + k];
      Lc[(size_t)i * n + j] = (i == j) ? std::sqrt(s) : s / Lc[(size_t)j * n + j];
    }
  // Li = L^{-1} (lower triangular)
  std::vector<double> Li((size_t)n * n, 0.0);
  for (int j = 0; j < n; ++j) {
    Li[(size_t)j * n + j] = 1.0 / Lc[(size_t)j * n + j];
    for (int i = j + 1; i < n; ++i) {
      double s = 0.0;
      for (int k = j; k < i; ++k) s -= Lc[(size_t)i * n + k] * Li[(size_t)k * n + j];
      Li[(size_t)i * n + j] = s / Lc[(size_t)i * n + i];
    }
  }
  // A = L^{-1} K L^{-T}
  std::vector<double> T((size_t)n * n, 0.0), A((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int k = 0; k <= i; ++k) s += Li[(size_t)i * n + k] * K[(size_t)k * n + j];
      T[(size_t)i * n + j] = s;
    }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int k = 0; k <= j; ++k) s += T[(size_t)i * n + k] * Li[(size_t)j * n + k];
      A[(size_t)i * n + j] = s;
    }
  for (int i = 0; i < n; ++i)   // exact symmetry before the rotations
    for (int j = i + 1; j < n; ++j) {
      const double s = 0.5 * (A[(size_t)i * n + j] + A[(size_t)j * n + i]);
      A[(size_t)i * n + j] = A[(size_t)j * n + i] = s;
    }
  std::vector<double> Q, l;
  jacobi_eigen(n, A, Q, l);
  std::vector<int> idx(n);
  for (int i = 0; i < n; ++i) idx[i] = i;
  std::sort(idx.begin(), idx.end(), [&](int p, int q) { return l[p] < l[q]; });
  // X = L^{-T} Q, columns in ascending Lambda
  X.assign((size_t)n * n, 0.0);
  lam.resize(n);
  for (int m = 0; m < n; ++m) {
    const int src = idx[m];
    lam[m] = l[src];
    for (int i = 0; i < n; ++i) {
      double s = 0.0;
      for (int k = i; k < n; ++k) s += Li[(size_t)k * n + i] * Q[(size_t)k * n + src];
      X[(size_t)i * n + m] = s;
    }
  }
  lam[0] = 0.0;   // the constant mode (zero up to rounding)
}

// ---------------------------------------------------------------------------
// kernels (FP64)
// ---------------------------------------------------------------------------

// rho_I(x_q) = sum_a Z_a e^{-r^2/s_a^2} / (pi^{3/2} s_a^3) over every periodic
// image within 6.8 s_a (where the Gaussian is below 1e-20)
__global__ void k_ion_density(int64_t nq, const double *__restrict__ x, int natoms,
                              const double *__restrict__ atoms, double ax, double ay, double az,
                              double *__restrict__ rho) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nq) return;
  const double av[3] = {ax, ay, az};
  double s = 0.0;
  for (int ia = 0; ia < natoms; ++ia) {
    const double *at = atoms + 5 * ia;
    const double sig = at[4], rc = 6.8 * sig;
    double d[3];
    int lo[3], hi[3];
    for (int k = 0; k < 3; ++k) {
      d[k] = x[3 * q + k] - at[k];
      lo[k] = (int)ceil((-rc - d[k]) / av[k]);
      hi[k] = (int)floor((rc - d[k]) / av[k]);
    }
    const double amp = at[3] / (PI * sqrt(PI) * sig * sig * sig), is2 = 1.0 / (sig * sig);
    for (int i = lo[0]; i <= hi[0]; ++i)
      for (int j = lo[1]; j <= hi[1]; ++j)
        for (int k = lo[2]; k <= hi[2]; ++k) {
          const double dx = d[0] + i * ax, dy = d[1] + j * ay, dz = d[2] + k * az;
          s += amp * exp(-(dx * dx + dy * dy + dz * dz) * is2);
        }
  }
  rho[q] = s;
}

constexpr int SCF_PMAX = 16;   // largest points per axis of a (sub)cell

// 1D Lagrange factors of one p^3 (sub)cell along its three axes:
// L1[(d * 4 + a) * SCF_PMAX + t] for axis d, function a, axis point t
__device__ __forceinline__ void cell_tables(const double *__restrict__ xi, int64_t qs, int p,
                                            double *L1) {
  for (int o = threadIdx.x; o < 3 * p; o += blockDim.x) {
    const int d = o / p, t = o - d * p;
    const int64_t stride = d == 0 ? 1 : (d == 1 ? p : (int64_t)p * p);
    double L[4], dL[4];
    lagrange3(xi[3 * (qs + t * stride) + d], L, dL);
    for (int a = 0; a < 4; ++a) L1[(d * 4 + a) * SCF_PMAX + t] = L[a];
  }
}

// b_i += scale sum_q w_q phi_i(x_q) f_q over the 64 FE functions of every
// element, by sum factorization over each p^3 (sub)cell (contract z, then
// y, then x: 4 p^3 + 16 p^2 + 64 p multiply-adds per cell)
__global__ void __launch_bounds__(128) k_fe_load(
    const int64_t *__restrict__ qoff, const double *__restrict__ w, const double *__restrict__ xi,
    const int32_t *__restrict__ partoff, const int32_t *__restrict__ part_p,
    const int32_t *__restrict__ part_q, const int64_t *__restrict__ doff,
    const int32_t *__restrict__ dofs, const double *__restrict__ f, double scale,
    double *__restrict__ b, unsigned *err) {
  __shared__ double L1[12 * SCF_PMAX];
  __shared__ double T1[SCF_PMAX * SCF_PMAX * 4];   // [qx + p qy][c]
  __shared__ double T2[SCF_PMAX * 16];             // [qx][b + 4 c]
  __shared__ double bl[64];
  const int e = blockIdx.x, tid = threadIdx.x;
  if (tid < 64) bl[tid] = 0.0;
  for (int k = partoff[e]; k < partoff[e + 1]; ++k) {
    const int p = part_p[k], p2 = p * p;
    if (p > SCF_PMAX) {
      if (tid == 0) atomicOr(err, DEVERR_SHAPE);
      return;
    }
    const int64_t qs = qoff[e] + part_q[k];
    __syncthreads();
    cell_tables(xi, qs, p, L1);
    __syncthreads();
    for (int it = tid; it < p2 * 4; it += blockDim.x) {   // z
      const int qxy = it >> 2, c = it & 3;
      double s = 0.0;
      for (int qz = 0; qz < p; ++qz) {
        const int64_t q = qs + qxy + (int64_t)p2 * qz;
        s += w[q] * f[q] * L1[(8 + c) * SCF_PMAX + qz];
      }
      T1[it] = s;
    }
    __syncthreads();
    for (int it = tid; it < p * 16; it += blockDim.x) {   // y
      const int qx = it >> 4, bc = it & 15, bb = bc & 3, c = bc >> 2;
      double s = 0.0;
      for (int qy = 0; qy < p; ++qy) s += T1[(qx + p * qy) * 4 + c] * L1[(4 + bb) * SCF_PMAX + qy];
      T2[it] = s;
    }
    __syncthreads();
    if (tid < 64) {                                       // x
      const int a = tid & 3, bc = tid >> 2;
      double s = 0.0;
      for (int qx = 0; qx < p; ++qx) s += T2[qx * 16 + bc] * L1[a * SCF_PMAX + qx];
      bl[tid] += s;
    }
  }
  __syncthreads();
  if (tid < 64) atomicAdd(b + dofs[doff[e] + tid], scale * bl[tid]);
}

// out = A applied along axis `axis` of the (n0, n1, n2) node array (x fastest):
// out[.., j, ..] = sum_k A[k][j] in[.., k, ..] (transpose = true: A^T, i.e.
// sum_k A[k][j]; transpose = false: sum_k A[j][k])
__global__ void k_axis(int n0, int n1, int n2, int axis, const double *__restrict__ A,
                       bool transpose, const double *__restrict__ in, double *__restrict__ out) {
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t total = (int64_t)n0 * n1 * n2;
  if (id >= total) return;
  const int i0 = (int)(id % n0), i1 = (int)((id / n0) % n1), i2 = (int)(id / ((int64_t)n0 * n1));
  const int n = axis == 0 ? n0 : (axis == 1 ? n1 : n2);
  const int j = axis == 0 ? i0 : (axis == 1 ? i1 : i2);
  const int64_t stride = axis == 0 ? 1 : (axis == 1 ? n0 : (int64_t)n0 * n1);
  const int64_t base = id - (int64_t)j * stride;
  double s = 0.0;
  for (int k = 0; k < n; ++k) {
    const double a = transpose ? A[(size_t)k * n + j] : A[(size_t)j * n + k];
    s += a * in[base + (int64_t)k * stride];
  }
  out[id] = s;
}

// c_abc /= (lx_a + ly_b + lz_c); the constant mode (0, 0, 0) -> 0
__global__ void k_modal_scale(int n0, int n1, int n2, const double *__restrict__ l0,
                              const double *__restrict__ l1, const double *__restrict__ l2,
                              double *__restrict__ c) {
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t total = (int64_t)n0 * n1 * n2;
  if (id >= total) return;
  const int i0 = (int)(id % n0), i1 = (int)((id / n0) % n1), i2 = (int)(id / ((int64_t)n0 * n1));
  c[id] = (id == 0) ? 0.0 : c[id] / (l0[i0] + l1[i1] + l2[i2]);
}

// V(x_q) = sum_i v_i phi_i(x_q) over the 64 FE functions, by sum
// factorization over each p^3 (sub)cell (x, then y, then z)
__global__ void __launch_bounds__(128) k_fe_interp(
    const int64_t *__restrict__ qoff, const double *__restrict__ xi,
    const int32_t *__restrict__ partoff, const int32_t *__restrict__ part_p,
    const int32_t *__restrict__ part_q, const int64_t *__restrict__ doff,
    const int32_t *__restrict__ dofs, const double *__restrict__ v, double *__restrict__ out,
    unsigned *err) {
  __shared__ double L1[12 * SCF_PMAX];
  __shared__ double ve[64];
  __shared__ double T1[16 * SCF_PMAX];              // [b + 4 c][qx]
  __shared__ double T2[4 * SCF_PMAX * SCF_PMAX];    // [c][qx + p qy]
  const int e = blockIdx.x, tid = threadIdx.x;
  if (tid < 64) ve[tid] = v[dofs[doff[e] + tid]];
  for (int k = partoff[e]; k < partoff[e + 1]; ++k) {
    const int p = part_p[k], p2 = p * p;
    if (p > SCF_PMAX) {
      if (tid == 0) atomicOr(err, DEVERR_SHAPE);
      return;
    }
    const int64_t qs = qoff[e] + part_q[k];
    __syncthreads();
    cell_tables(xi, qs, p, L1);
    __syncthreads();
    for (int it = tid; it < 16 * p; it += blockDim.x) {   // x
      const int bc = it / p, qx = it - bc * p;
      double s = 0.0;
      for (int a = 0; a < 4; ++a) s += ve[a + 4 * bc] * L1[a * SCF_PMAX + qx];
      T1[it] = s;
    }
    __syncthreads();
    for (int it = tid; it < 4 * p2; it += blockDim.x) {   // y
      const int c = it / p2, qxy = it - c * p2, qy = qxy / p, qx = qxy - qy * p;
      double s = 0.0;
      for (int bb = 0; bb < 4; ++bb) s += T1[(bb + 4 * c) * p + qx] * L1[(4 + bb) * SCF_PMAX + qy];
      T2[it] = s;
    }
    __syncthreads();
    for (int it = tid; it < p2 * p; it += blockDim.x) {   // z
      const int qz = it / p2, qxy = it - qz * p2;
      double s = 0.0;
      for (int c = 0; c < 4; ++c) s += T2[c * p2 + qxy] * L1[(8 + c) * SCF_PMAX + qz];
      out[qs + it] = s;
    }
  }
}

// Dirac exchange + Perdew-Zunger 1981 correlation (unpolarised); 0 for n <= 1e-30
__device__ inline void lda_pz81(double n, double &e, double &v) {
  if (!(n > 1e-30)) {
    e = v = 0.0;
    return;
  }
  const double rs = cbrt(3.0 / (4.0 * PI * n));
  const double ex = -0.75 * cbrt(3.0 * n / PI);
  double ec, vc;
  if (rs >= 1.0) {
    const double sq = sqrt(rs), den = 1.0 + 1.0529 * sq + 0.3334 * rs;
    ec = -0.1423 / den;
    vc = ec * (1.0 + 7.0 / 6.0 * 1.0529 * sq + 4.0 / 3.0 * 0.3334 * rs) / den;
  } else {
    const double lr = log(rs);
    ec = 0.0311 * lr - 0.048 + 0.0020 * rs * lr - 0.0116 * rs;
    vc = 0.0311 * lr + (-0.048 - 0.0311 / 3.0) + 2.0 / 3.0 * 0.0020 * rs * lr +
         (2.0 * -0.0116 - 0.0020) / 3.0 * rs;
  }
  e = ex + ec;
  v = 4.0 / 3.0 * ex + vc;
}

__global__ void k_xc(int64_t nq, const double *__restrict__ n, double *__restrict__ exc,
                     double *__restrict__ vxc) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nq) return;
  double e, v;
  lda_pz81(n[q], e, v);
  if (exc) exc[q] = e;
  if (vxc) vxc[q] = v;
}

__global__ void k_diff(int64_t nq, const double *__restrict__ a, const double *__restrict__ b,
                       double *__restrict__ out) {   // out = a - b
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < nq) out[q] = a[q] - b[q];
}

__global__ void k_add(int64_t nq, const double *__restrict__ a, const double *__restrict__ b,
                      double *__restrict__ out) {    // out = a + b
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < nq) out[q] = a[q] + b[q];
}

// energies of n_out and the residual, one pass over the points:
// sums[0] += w n_out V_in, sums[1] += w (rho_I - n_out) V_C, sums[2] += w n_out eps_xc,
// sums[3] += w |n_out - n_in|; then n_in <- n_in + alpha (n_out - n_in)
__global__ void k_energy_mix(int64_t nq, const double *__restrict__ w, const double *__restrict__ n_out,
                             const double *__restrict__ V_in, const double *__restrict__ rho_I,
                             const double *__restrict__ vc, const double *__restrict__ exc,
                             double alpha, double *__restrict__ n_in, double *__restrict__ sums) {
  __shared__ double red[4][32];
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double s[4] = {0.0, 0.0, 0.0, 0.0};
  if (q < nq) {
    const double no = n_out[q], wq = w[q], ni = n_in[q];
    s[0] = wq * no * V_in[q];
    s[1] = wq * (rho_I[q] - no) * vc[q];
    s[2] = wq * no * exc[q];
    s[3] = wq * fabs(no - ni);
    n_in[q] = ni + alpha * (no - ni);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = 0; k < 4; ++k) {
    double t = s[k];
    for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
    if (lane == 0) red[k][warp] = t;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[threadIdx.x][i];
    atomicAdd(sums + threadIdx.x, t);
  }
}

constexpr int PULAY_MAX = 8;
struct SlotList {
  int m;
  int s[PULAY_MAX];
  double c[PULAY_MAX];
};

// store (n_in, n_out - n_in) in slot `slot` of the history and accumulate
// dots[j] += sum_q w_q R_new R_j for the active slots
__global__ void k_pulay_store(int64_t nq, const double *__restrict__ w,
                              const double *__restrict__ n_in, const double *__restrict__ n_out,
                              int slot, SlotList L, double *__restrict__ hn, double *__restrict__ hR,
                              double *__restrict__ dots) {
  __shared__ double red[PULAY_MAX][8];
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double r = 0.0, wq = 0.0;
  if (q < nq) {
    r = n_out[q] - n_in[q];
    wq = w[q];
    hn[(int64_t)slot * nq + q] = n_in[q];
    hR[(int64_t)slot * nq + q] = r;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int j = 0; j < L.m; ++j) {
    double t = 0.0;
    if (q < nq) t = wq * r * (L.s[j] == slot ? r : hR[(int64_t)L.s[j] * nq + q]);
    for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
    if (lane == 0) red[j][warp] = t;
  }
  __syncthreads();
  if (threadIdx.x < L.m) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[threadIdx.x][i];
    atomicAdd(dots + threadIdx.x, t);
  }
}

// n = sum_i c_i (n_i + alpha R_i) over the active slots
__global__ void k_pulay_mix(int64_t nq, SlotList L, double alpha, const double *__restrict__ hn,
                            const double *__restrict__ hR, double *__restrict__ n) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nq) return;
  double s = 0.0;
  for (int i = 0; i < L.m; ++i)
    s += L.c[i] * (hn[(int64_t)L.s[i] * nq + q] + alpha * hR[(int64_t)L.s[i] * nq + q]);
  n[q] = s;
}

// solve the (m + 1) bordered system [A 1; 1^T 0] [c; l] = [0; 1] by Gaussian
// elimination with partial pivoting (m <= 8)
static bool pulay_coefficients(int m, const double A[8][8], double *c) {
  double M[9][10] = {{0}};
  double tr = 0.0;
  for (int i = 0; i < m; ++i) tr += A[i][i];
  const double ridge = 1e-12 * tr / m;
  for (int i = 0; i < m; ++i) {
    for (int j = 0; j < m; ++j) M[i][j] = A[i][j] + (i == j ? ridge : 0.0);
    M[i][m] = 1.0;
    M[m][i] = 1.0;
  }
  M[m][m + 1] = 1.0;
  const int n = m + 1;
  for (int k = 0; k < n; ++k) {
    int piv = k;
    for (int i = k + 1; i < n; ++i)
      if (std::fabs(M[i][k]) > std::fabs(M[piv][k])) piv = i;
    if (std::fabs(M[piv][k]) < 1e-300) return false;
    for (int j = 0; j <= n; ++j) std::swap(M[k][j], M[piv][j]);
    for (int i = k + 1; i < n; ++i) {
      const double f = M[i][k] / M[k][k];
      for (int j = k; j <= n; ++j) M[i][j] -= f * M[k][j];
    }
  }
  double x[9];
  for (int i = n - 1; i >= 0; --i) {
    double t = M[i][n];
    for (int j = i + 1; j < n; ++j) t -= M[i][j] * x[j];
    x[i] = t / M[i][i];
  }
  for (int i = 0; i < m; ++i) c[i] = x[i];
  return true;
}

inline unsigned blocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

pufe_status scf_prepare(pufe_ctx *ctx) {
  if (ctx->scf) return PUFE_OK;
  if (ctx->max_part_p > SCF_PMAX) return fail(PUFE_EINVAL, "rule with more than 16 points per axis");
  auto *S = new ScfState();
  ctx->scf = S;
  auto &D = ctx->d;
  (void)D;
  for (int d = 0; d < 3; ++d) {
    std::vector<double> X, lam;
    axis_modes(ctx->nel[d], ctx->h[d], X, lam);
    S->n1[d] = 3 * ctx->nel[d];
    PUFE_CUDA_TRY(cudaMalloc((void **)&S->X[d], X.size() * sizeof(double)));
    PUFE_CUDA_TRY(cudaMalloc((void **)&S->lam[d], lam.size() * sizeof(double)));
    PUFE_CUDA_TRY(cudaMemcpy(S->X[d], X.data(), X.size() * sizeof(double), cudaMemcpyHostToDevice));
    PUFE_CUDA_TRY(
        cudaMemcpy(S->lam[d], lam.data(), lam.size() * sizeof(double), cudaMemcpyHostToDevice));
  }
  const size_t nfe = (size_t)ctx->n_fe * sizeof(double), nq = (size_t)ctx->nq * sizeof(double);
  PUFE_CUDA_TRY(cudaMalloc((void **)&S->b, nfe));
  PUFE_CUDA_TRY(cudaMalloc((void **)&S->t0, nfe));
  PUFE_CUDA_TRY(cudaMalloc((void **)&S->t1, nfe));
  PUFE_CUDA_TRY(cudaMalloc((void **)&S->n_out, nq));
  PUFE_CUDA_TRY(cudaMalloc((void **)&S->vc, nq));
  PUFE_CUDA_TRY(cudaMalloc((void **)&S->exc, nq));
  PUFE_CUDA_TRY(cudaMalloc((void **)&S->vxc, nq));
  PUFE_CUDA_TRY(cudaMalloc((void **)&S->sums, 8 * sizeof(double)));
  PUFE_CUDA_TRY(cudaMalloc((void **)&S->f, 64 * 64 * sizeof(double)));
  return PUFE_OK;
}

void scf_free(pufe_ctx *ctx) {
  ScfState *S = ctx->scf;
  if (!S) return;
  void *ptrs[] = {S->X[0], S->X[1], S->X[2], S->lam[0], S->lam[1], S->lam[2], S->b, S->t0,
                  S->t1, S->n_out, S->vc, S->exc, S->vxc, S->sums, S->f, S->nk, S->atoms,
                  S->hist_n, S->hist_R, S->dots};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  delete S;
  ctx->scf = nullptr;
}

pufe_status launch_ion_density(pufe_ctx *ctx, int natoms, const double *tau, const double *Z,
                               const double *sigma, double *rho, cudaStream_t st) {
  if (pufe_status e0 = scf_prepare(ctx)) return e0;
  ScfState *S = ctx->scf;
  if (natoms > S->atoms_cap) {
    if (S->atoms) PUFE_CUDA_TRY(cudaFree(S->atoms));
    S->atoms = nullptr;
    PUFE_CUDA_TRY(cudaMalloc((void **)&S->atoms, (size_t)5 * std::max(1, natoms) * sizeof(double)));
    S->atoms_cap = natoms;
  }
  std::vector<double> at((size_t)5 * std::max(1, natoms), 0.0);
  double es = 0.0;
  for (int a = 0; a < natoms; ++a) {
    for (int k = 0; k < 3; ++k) at[5 * a + k] = tau[3 * a + k];
    at[5 * a + 3] = Z[a];
    at[5 * a + 4] = sigma[a];
    es += Z[a] * Z[a] / (sigma[a] * std::sqrt(2.0 * PI));
  }
  S->e_self = es;
  // synchronous copy: the host vector is a temporary
  PUFE_CUDA_TRY(cudaMemcpy(S->atoms, at.data(), at.size() * sizeof(double), cudaMemcpyHostToDevice));
  k_ion_density<<<blocks(ctx->nq, 256), 256, 0, st>>>(ctx->nq, ctx->d.x, natoms, S->atoms,
                                                      ctx->a[0], ctx->a[1], ctx->a[2], rho);
  PUFE_CUDA_TRY(cudaGetLastError());
  return PUFE_OK;
}

// V_C with del^2 V_C = 4 pi (rho_I - n), zero cell average, at the points
static pufe_status coulomb(pufe_ctx *ctx, const double *n, const double *rho_I, double *VC,
                           cudaStream_t st) {
  ScfState *S = ctx->scf;
  auto &D = ctx->d;
  const int n0 = S->n1[0], n1 = S->n1[1], n2 = S->n1[2];
  const int64_t nfe = ctx->n_fe;
  // f = n - rho_I at the points (in vc as scratch), b = int phi f
  k_diff<<<blocks(ctx->nq, 256), 256, 0, st>>>(ctx->nq, n, rho_I, VC);
  PUFE_CUDA_TRY(cudaMemsetAsync(S->b, 0, nfe * sizeof(double), st));
  // -K v = 4 pi int phi (rho_I - n)  <=>  K v = 4 pi int phi (n - rho_I)
  k_fe_load<<<(unsigned)ctx->nelem, 128, 0, st>>>(D.qoff, D.w, D.xi, D.partoff, D.part_p,
                                                  D.part_q, D.doff, D.dofs, VC, 4.0 * PI, S->b,
                                                  D.err);
  const unsigned nb = blocks(nfe, 256);
  k_axis<<<nb, 256, 0, st>>>(n0, n1, n2, 0, S->X[0], true, S->b, S->t0);
  k_axis<<<nb, 256, 0, st>>>(n0, n1, n2, 1, S->X[1], true, S->t0, S->t1);
  k_axis<<<nb, 256, 0, st>>>(n0, n1, n2, 2, S->X[2], true, S->t1, S->t0);
  k_modal_scale<<<nb, 256, 0, st>>>(n0, n1, n2, S->lam[0], S->lam[1], S->lam[2], S->t0);
  k_axis<<<nb, 256, 0, st>>>(n0, n1, n2, 2, S->X[2], false, S->t0, S->t1);
  k_axis<<<nb, 256, 0, st>>>(n0, n1, n2, 1, S->X[1], false, S->t1, S->t0);
  k_axis<<<nb, 256, 0, st>>>(n0, n1, n2, 0, S->X[0], false, S->t0, S->t1);
  k_fe_interp<<<(unsigned)ctx->nelem, 128, 0, st>>>(D.qoff, D.xi, D.partoff, D.part_p,
                                                    D.part_q, D.doff, D.dofs, S->t1, VC, D.err);
  PUFE_CUDA_TRY(cudaGetLastError());
  return PUFE_OK;
}

pufe_status launch_effective_potential(pufe_ctx *ctx, const double *n, const double *rho_I,
                                       double *V_eff, double *V_C, double *eps_xc,
                                       cudaStream_t st) {
  if (pufe_status e0 = scf_prepare(ctx)) return e0;
  ScfState *S = ctx->scf;
  double *vc = V_C ? V_C : S->vc;
  if (pufe_status e1 = coulomb(ctx, n, rho_I, vc, st)) return e1;
  k_xc<<<blocks(ctx->nq, 256), 256, 0, st>>>(ctx->nq, n, eps_xc, S->vxc);
  k_add<<<blocks(ctx->nq, 256), 256, 0, st>>>(ctx->nq, vc, S->vxc, V_eff);
  PUFE_CUDA_TRY(cudaGetLastError());
  return PUFE_OK;
}

void scf_reset(pufe_ctx *ctx) {
  if (!ctx->scf) return;
  ctx->scf->slots.clear();
  ctx->scf->next_slot = 0;
}

// Fermi-Dirac occupations of nk k-points x nstates states (eps and f
// k-major) with weights wk (nullptr: one k-point of weight 1): mu by bisection
// on sum_k w_k sum_n f_nk = nelec; the band energy and the entropy sum
// sum_k w_k sum_n [g ln g + (1 - g) ln(1 - g)] (g = f / 2) weighted alike.
static double occupations(int nk, const double *wk, int nstates, const double *eps, double nelec,
                          double kT, std::vector<double> &f, double &e_band, double &ts) {
  const int nt = nk * nstates;
  double lo = eps[0], hi = eps[0];
  for (int k = 1; k < nt; ++k) {
    lo = std::min(lo, eps[k]);
    hi = std::max(hi, eps[k]);
  }
  lo -= 50.0 * kT + 1.0;
  hi += 50.0 * kT + 1.0;
  f.assign(nt, 0.0);
  auto occ = [&](double mu) {
    double s = 0.0;
    for (int k = 0; k < nt; ++k) {
      const double x = std::min(700.0, std::max(-700.0, (eps[k] - mu) / kT));
      f[k] = 2.0 / (1.0 + std::exp(x));
      s += (wk ? wk[k / nstates] : 1.0) * f[k];
    }
    return s;
  };
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (occ(mid) < nelec)
      lo = mid;
    else
      hi = mid;
  }
  const double mu = 0.5 * (lo + hi);
  occ(mu);
  e_band = 0.0;
  ts = 0.0;
  for (int k = 0; k < nt; ++k) {
    const double w = wk ? wk[k / nstates] : 1.0;
    e_band += w * f[k] * eps[k];
    const double g = f[k] / 2.0;
    if (g > 1e-300 && g < 1.0 - 1e-16) ts += w * (g * std::log(g) + (1.0 - g) * std::log1p(-g));
  }
  ts *= -2.0;
  return mu;
}

static pufe_status scf_finish(pufe_ctx *ctx, double mu, double e_band, double ts, double kT,
                              double alpha, int pulay, const double *rho_I,
                              const double *V_eff_in, double *n, double *V_eff_out,
                              pufe_scf_info *info, cudaStream_t st);

pufe_status launch_scf_step(pufe_ctx *ctx, int nstates, const double *eps, const double *C,
                            int64_t ldc, double nelec, double kT, double alpha, int pulay, int prec,
                            const double *rho_I, const double *V_eff_in, double *n, double *V_eff_out,
                            double *f_out, pufe_scf_info *info, cudaStream_t st) {
  if (pufe_status e0 = scf_prepare(ctx)) return e0;
  ScfState *S = ctx->scf;
  std::vector<double> f;
  double e_band = 0.0, ts = 0.0;
  const double mu = occupations(1, nullptr, nstates, eps, nelec, kT, f, e_band, ts);
  if (f_out) std::copy(f.begin(), f.end(), f_out);
  PUFE_CUDA_TRY(cudaMemcpyAsync(S->f, f.data(), nstates * sizeof(double), cudaMemcpyHostToDevice, st));
  pufe_status e1 = (prec == PUFE_FP64)
                       ? launch_density_fp64(ctx, C, ldc, S->f, nstates, S->n_out, st)
                       : launch_density_tc(ctx, C, ldc, S->f, nstates, S->n_out, st);
  if (e1 != PUFE_OK) return e1;
  return scf_finish(ctx, mu, e_band, ts, kT, alpha, pulay, rho_I, V_eff_in, n, V_eff_out, info, st);
}

pufe_status launch_scf_step_bloch(pufe_ctx *ctx, int nk, const double *kpts, const double *wk,
                                  int nstates, const double *eps, const double *const *C_re,
                                  const double *const *C_im, int64_t ldc, double nelec, double kT,
                                  double alpha, int pulay, int prec, const double *rho_I,
                                  const double *V_eff_in, double *n, double *V_eff_out,
                                  double *f_out, pufe_scf_info *info, cudaStream_t st) {
  if (pufe_status e0 = scf_prepare(ctx)) return e0;
  ScfState *S = ctx->scf;
  if (!S->nk) PUFE_CUDA_TRY(cudaMalloc((void **)&S->nk, (size_t)ctx->nq * sizeof(double)));
  std::vector<double> f;
  double e_band = 0.0, ts = 0.0;
  const double mu = occupations(nk, wk, nstates, eps, nelec, kT, f, e_band, ts);
  if (f_out) std::copy(f.begin(), f.end(), f_out);
  // n_out = sum_k w_k sum_n f_nk |psi_nk|^2: each k's density with the
  // occupations w_k f_nk, added into n_out
  std::vector<double> fw(f.size());
  for (size_t i = 0; i < f.size(); ++i) fw[i] = wk[i / nstates] * f[i];
  PUFE_CUDA_TRY(cudaMemcpyAsync(S->f, fw.data(), fw.size() * sizeof(double), cudaMemcpyHostToDevice,
                                st));
  for (int i = 0; i < nk; ++i) {
    const PhaseTab ph = phase_table(ctx, kpts + 3 * i);
    double *out = i == 0 ? S->n_out : S->nk;
    const double *fk = S->f + (size_t)i * nstates;
    pufe_status e1 = (prec == PUFE_FP64)
                         ? launch_density_fp64_bloch(ctx, ph, C_re[i], C_im[i], ldc, fk, nstates,
                                                     out, st)
                         : launch_density_tc(ctx, C_re[i], ldc, fk, nstates, out, st, C_im[i], &ph);
    if (e1 != PUFE_OK) return e1;
    if (i > 0) {
      k_add<<<blocks(ctx->nq, 256), 256, 0, st>>>(ctx->nq, S->n_out, S->nk, S->n_out);
      PUFE_CUDA_TRY(cudaGetLastError());
    }
  }
  return scf_finish(ctx, mu, e_band, ts, kT, alpha, pulay, rho_I, V_eff_in, n, V_eff_out, info, st);
}

// the part of an SCF step after the output density S->n_out: V_C[n_out] and
// eps_xc(n_out), the energies, mixing into n and the new potential
static pufe_status scf_finish(pufe_ctx *ctx, double mu, double e_band, double ts, double kT,
                              double alpha, int pulay, const double *rho_I,
                              const double *V_eff_in, double *n, double *V_eff_out,
                              pufe_scf_info *info, cudaStream_t st) {
  ScfState *S = ctx->scf;
  if (pufe_status e2 = coulomb(ctx, S->n_out, rho_I, S->vc, st)) return e2;
  k_xc<<<blocks(ctx->nq, 256), 256, 0, st>>>(ctx->nq, S->n_out, S->exc, nullptr);
  PUFE_CUDA_TRY(cudaMemsetAsync(S->sums, 0, 8 * sizeof(double), st));
  const bool use_pulay = pulay > 1;
  k_energy_mix<<<blocks(ctx->nq, 256), 256, 0, st>>>(ctx->nq, ctx->d.w, S->n_out, V_eff_in, rho_I,
                                                     S->vc, S->exc, use_pulay ? 0.0 : alpha, n,
                                                     S->sums);
  PUFE_CUDA_TRY(cudaGetLastError());
  if (use_pulay) {
    const int depth = std::min(pulay, PULAY_MAX);
    if (!S->hist_n) {
      PUFE_CUDA_TRY(cudaMalloc((void **)&S->hist_n, (size_t)PULAY_MAX * ctx->nq * sizeof(double)));
      PUFE_CUDA_TRY(cudaMalloc((void **)&S->hist_R, (size_t)PULAY_MAX * ctx->nq * sizeof(double)));
      PUFE_CUDA_TRY(cudaMalloc((void **)&S->dots, PULAY_MAX * sizeof(double)));
    }
    // drop the oldest entries beyond depth - 1, then add this one
    while ((int)S->slots.size() > depth - 1) S->slots.erase(S->slots.begin());
    int slot = 0;
    while (std::find(S->slots.begin(), S->slots.end(), slot) != S->slots.end()) ++slot;
    S->slots.push_back(slot);
    SlotList L;
    L.m = (int)S->slots.size();
    for (int i = 0; i < L.m; ++i) L.s[i] = S->slots[i];
    PUFE_CUDA_TRY(cudaMemsetAsync(S->dots, 0, PULAY_MAX * sizeof(double), st));
    k_pulay_store<<<blocks(ctx->nq, 256), 256, 0, st>>>(ctx->nq, ctx->d.w, n, S->n_out, slot, L,
                                                        S->hist_n, S->hist_R, S->dots);
    PUFE_CUDA_TRY(cudaGetLastError());
    double dots[PULAY_MAX];
    PUFE_CUDA_TRY(cudaMemcpyAsync(dots, S->dots, L.m * sizeof(double), cudaMemcpyDeviceToHost, st));
    PUFE_CUDA_TRY(cudaStreamSynchronize(st));
    for (int j = 0; j < L.m; ++j) S->gram[slot][L.s[j]] = S->gram[L.s[j]][slot] = dots[j];
    double A[8][8];
    for (int i = 0; i < L.m; ++i)
      for (int j = 0; j < L.m; ++j) A[i][j] = S->gram[L.s[i]][L.s[j]];
    if (!pulay_coefficients(L.m, A, L.c)) return fail(PUFE_EINVAL, "Pulay system is singular");
    k_pulay_mix<<<blocks(ctx->nq, 256), 256, 0, st>>>(ctx->nq, L, alpha, S->hist_n, S->hist_R, n);
    PUFE_CUDA_TRY(cudaGetLastError());
  }
  // the new effective potential of the mixed density
  if (pufe_status e3 = launch_effective_potential(ctx, n, rho_I, V_eff_out, nullptr, nullptr, st))
    return e3;
  double sums[4];
  PUFE_CUDA_TRY(cudaMemcpyAsync(sums, S->sums, 4 * sizeof(double), cudaMemcpyDeviceToHost, st));
  PUFE_CUDA_TRY(cudaStreamSynchronize(st));
  if (info) {
    info->mu = mu;
    info->e_band = e_band;
    info->e_dc = -sums[0];
    info->e_es = -0.5 * sums[1];
    info->e_self = S->e_self;
    info->e_xc = sums[2];
    info->e_ts = -kT * ts;
    info->e_total = info->e_band + info->e_dc + info->e_es - info->e_self + info->e_xc + info->e_ts;
    info->residual = sums[3];
  }
  return PUFE_OK;
}

}  // namespace pufe
