// Host-side setup of the PUFE context: mesh, enrichment sets, per-element
// basis lists, quadrature rules, CSR pattern and scatter maps (runs once per
// geometry), plus the getters, error reporting and teardown of the C ABI.
//
// Paper map: basis of Sec. 4 (eqs. pufebasis, psih); enriched vertex sets
// and periodic enrichments of Sec. 5.1 (eq. Psi); quadrature of Sec. 5.2.
#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstring>
#include <functional>
#include <numeric>
#include <thread>

#include "pufe_internal.h"

namespace pufe {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

pufe_status fail(pufe_status st, const std::string &msg) {
  g_last_error = msg;
  return st;
}

pufe_status cuda_fail(cudaError_t err, const char *what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(err);
  return err == cudaErrorMemoryAllocation ? PUFE_ENOMEM : PUFE_ECUDA;
}

// ---------------------------------------------------------------------------
// Gauss-Legendre nodes/weights on [-1, 1] by Newton iteration on P_p.
// ---------------------------------------------------------------------------
static void gauss_legendre(int p, std::vector<double> &x, std::vector<double> &w) {
  x.assign(p, 0.0);
  w.assign(p, 0.0);
  const double PI = 3.14159265358979323846;
  for (int i = 0; i < p; ++i) {
    double t = std::cos(PI * (i + 0.75) / (p + 0.5));
    double dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = t;
      for (int k = 2; k <= p; ++k) {
        double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      if (p == 1) { p1 = t; p0 = 1.0; }
      dp = p * (t * p1 - p0) / (t * t - 1.0);
      double dt = p1 / dp;
      t -= dt;
      if (std::fabs(dt) < 1e-16) break;
    }
    // final derivative at the converged node
    double p0 = 1.0, p1 = t;
    for (int k = 2; k <= p; ++k) {
      double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    if (p == 1) { p1 = t; p0 = 1.0; }
    dp = p * (t * p1 - p0) / (t * t - 1.0);
    x[p - 1 - i] = t;  // ascending order
    w[p - 1 - i] = 2.0 / ((1.0 - t * t) * dp * dp);
  }
}

struct Box {
  double lo[3], hi[3];
};

struct RulePart {  // one tensor rule on one (sub)cell
  Box box;
  int p;
};

struct Setup {
  double a[3], h[3];
  int nel[3];
  int img[3];
  // general (triclinic) cell: element e maps the reference cube by
  // x = x0(e) + J (xi + 1), J = [a_d / 2 nel_d] (columns), |det J| = detJ
  bool gen = false;
  LatticeDev lat;        // rows a_d, L^-T, image half-widths
  double J[9], Jit[9];   // J (row-major, J[3 r + c]) and J^-T
  double detJ = 0.0;
  std::vector<Orbital> orb;          // alpha list
  std::vector<int> orb_atom;         // alpha -> atom
  std::vector<std::array<double, 3>> tau;
  std::vector<int> atom_species;
  std::vector<double> rc_species, re_species;
  std::vector<std::vector<double>> gx, gw;  // Gauss tables by order (index p)
};

static double box_point_dist(const Box &b, const double p[3]) {
  double s = 0.0;
  for (int k = 0; k < 3; ++k) {
    double d = std::max(std::max(b.lo[k] - p[k], p[k] - b.hi[k]), 0.0);
    s += d * d;
  }
  return std::sqrt(s);
}

// Distance from point P to the parallelepiped {x0 + M t : t in [0, 1]^3}
// (M row-major, columns the edges).  The squared distance is convex in t;
// its minimiser lies in the relative interior of one of the box's 27 faces
// (each coordinate free, at 0 or at 1).  Each face's free coordinates solve
// the normal equations of a least-squares problem (Cramer's rule, at most
// 3 x 3); feasible face minimisers are points of the parallelepiped, and the
// nearest of them is the exact answer.
static double parallelepiped_point_dist(const double x0[3], const double M[9], const double P[3]) {
  double best = 1e300;
  for (int code = 0; code < 27; ++code) {
    int st[3] = {code % 3, (code / 3) % 3, code / 9};   // 0 free, 1 at 0, 2 at 1
    int fr[3], nf = 0;
    double base[3] = {x0[0], x0[1], x0[2]};
    for (int d = 0; d < 3; ++d) {
      if (st[d] == 0) fr[nf++] = d;
      else if (st[d] == 2)
        for (int r = 0; r < 3; ++r) base[r] += M[3 * r + d];
    }
    double rv[3] = {P[0] - base[0], P[1] - base[1], P[2] - base[2]};
    double t[3] = {0, 0, 0};
    bool ok = true;
    if (nf > 0) {
      double G[3][3], g[3];
      for (int i = 0; i < nf; ++i) {
        g[i] = 0.0;
        for (int r = 0; r < 3; ++r) g[i] += M[3 * r + fr[i]] * rv[r];
        for (int j = 0; j < nf; ++j) {
          G[i][j] = 0.0;
          for (int r = 0; r < 3; ++r) G[i][j] += M[3 * r + fr[i]] * M[3 * r + fr[j]];
        }
      }
      double sol[3];
      if (nf == 1) {
        sol[0] = g[0] / G[0][0];
      } else if (nf == 2) {
        const double det = G[0][0] * G[1][1] - G[0][1] * G[1][0];
        sol[0] = (g[0] * G[1][1] - G[0][1] * g[1]) / det;
        sol[1] = (G[0][0] * g[1] - g[0] * G[1][0]) / det;
      } else {
        const double det = G[0][0] * (G[1][1] * G[2][2] - G[1][2] * G[2][1]) -
                           G[0][1] * (G[1][0] * G[2][2] - G[1][2] * G[2][0]) +
                           G[0][2] * (G[1][0] * G[2][1] - G[1][1] * G[2][0]);
        for (int c = 0; c < 3; ++c) {
          double A[3][3];
          for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) A[i][j] = j == c ? g[i] : G[i][j];
          sol[c] = (A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) -
                    A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
                    A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0])) / det;
        }
      }
      for (int i = 0; i < nf; ++i) {
        ok = ok && sol[i] >= 0.0 && sol[i] <= 1.0;
        t[fr[i]] = sol[i];
      }
    }
    if (!ok) continue;
    double q2 = 0.0;
    for (int r = 0; r < 3; ++r) {
      double x = base[r] - P[r];
      for (int i = 0; i < nf; ++i) x += M[3 * r + fr[i]] * t[fr[i]];
      q2 += x * x;
    }
    best = std::min(best, std::sqrt(q2));
  }
  return best;
}

// corner x0 of element (ex, ey, ez) of a general cell: L^T (e / nel)
static void elem_origin(const Setup &S, const int idx[3], double x0[3]) {
  for (int r = 0; r < 3; ++r) {
    x0[r] = 0.0;
    for (int d = 0; d < 3; ++d) x0[r] += (double)idx[d] / S.nel[d] * S.lat.L[3 * d + r];
  }
}

// smallest distance from any periodic image of atom position t to box b
static double atom_box_dist(const Setup &S, const double t[3], const Box &b) {
  double best = 1e300;
  const int R = 2;
  for (int i = -R; i <= R; ++i)
    for (int j = -R; j <= R; ++j)
      for (int k = -R; k <= R; ++k) {
        double p[3] = {t[0] + i * S.a[0], t[1] + j * S.a[1], t[2] + k * S.a[2]};
        best = std::min(best, box_point_dist(b, p));
      }
  return best;
}

// integrals of Psi^2 and |grad Psi|^2 on a box with the p^3 Gauss rule,
// for each alpha of `alphas`: out[2*i], out[2*i+1]
// (general cells: b is a box of the reference cube of the element with
// corner x0, mapped by J)
static void box_integrals(Setup &S, const std::vector<int> &alphas, const Box &b, int p,
                          std::vector<double> &out, const double *x0 = nullptr) {
  out.assign(2 * alphas.size(), 0.0);
  const std::vector<double> &gx = S.gx[p], &gw = S.gw[p];
  double half[3], mid[3];
  for (int k = 0; k < 3; ++k) {
    half[k] = 0.5 * (b.hi[k] - b.lo[k]);
    mid[k] = 0.5 * (b.hi[k] + b.lo[k]);
  }
  for (size_t ia = 0; ia < alphas.size(); ++ia) {
    const Orbital &o = S.orb[alphas[ia]];
    double s0 = 0.0, s1 = 0.0;
    for (int kz = 0; kz < p; ++kz)
      for (int ky = 0; ky < p; ++ky)
        for (int kx = 0; kx < p; ++kx) {
          double pt[3] = {mid[0] + half[0] * gx[kx], mid[1] + half[1] * gx[ky],
                          mid[2] + half[2] * gx[kz]};
          double wt = gw[kx] * gw[ky] * gw[kz] * half[0] * half[1] * half[2];
          double psi, g[3];
          if (S.gen) {
            double x[3];
            for (int r = 0; r < 3; ++r)
              x[r] = x0[r] + S.J[3 * r] * (pt[0] + 1.0) + S.J[3 * r + 1] * (pt[1] + 1.0) +
                     S.J[3 * r + 2] * (pt[2] + 1.0);
            enrichment_eval_lat(o, x, S.lat, psi, g);
            wt *= S.detJ;
          } else {
            enrichment_eval(o, pt, S.a, S.img, psi, g);
          }
          s0 += wt * psi * psi;
          s1 += wt * (g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
        }
    out[2 * ia] = s0;
    out[2 * ia + 1] = s1;
  }
}

static void hadapt(Setup &S, const std::vector<int> &alphas, const Box &b, int depth,
                   const pufe_quad &q, std::vector<RulePart> &parts, const double *x0) {
  std::vector<double> i5, i8;
  box_integrals(S, alphas, b, 5, i5, x0);
  box_integrals(S, alphas, b, 8, i8, x0);
  std::vector<int> failing;
  for (size_t ia = 0; ia < alphas.size(); ++ia)
    if (std::fabs(i5[2 * ia] - i8[2 * ia]) >= q.tol ||
        std::fabs(i5[2 * ia + 1] - i8[2 * ia + 1]) >= q.tol)
      failing.push_back(alphas[ia]);
  if (failing.empty() || depth >= q.max_depth) {
    parts.push_back({b, 8});
    return;
  }
  double mid[3];
  for (int k = 0; k < 3; ++k) mid[k] = 0.5 * (b.lo[k] + b.hi[k]);
  for (int c = 0; c < 2; ++c)
    for (int bb = 0; bb < 2; ++bb)
      for (int a = 0; a < 2; ++a) {
        int off[3] = {a, bb, c};
        Box ch;
        for (int k = 0; k < 3; ++k) {
          ch.lo[k] = off[k] == 0 ? b.lo[k] : mid[k];
          ch.hi[k] = off[k] == 0 ? mid[k] : b.hi[k];
        }
        hadapt(S, failing, ch, depth + 1, q, parts, x0);
      }
}

// ---- the adaptive tests on the GPU (Sec. 5.2) ---------------------------------
// One test is the pair of integrals I(Psi^2), I(|grad Psi|^2) of one
// enrichment on one box with the p^3 Gauss rule, exactly as box_integrals
// forms them on the host (same points, weights and integrands); the tests of
// a whole level of the adaptive construction run as one launch, one CTA per
// test, each thread summing a strided subset of the points and the CTA
// reducing them in a fixed tree order.  The decisions (which p, which
// integrands fail, which cells split) stay with the host, on these values.
struct RuleTest {
  double lo[3], hi[3];   // box (reference cube of the element for general cells)
  double x0[3];          // element corner (general cells)
  int alpha, p;
};

struct Jmat {
  double m[9];
};

constexpr int RT_NT = 128;
constexpr int RT_PMAX = 18;   // largest Gauss order of the tests (PADAPT reads p_max + 2)

__global__ void __launch_bounds__(RT_NT) k_rule_tests(
    const RuleTest *__restrict__ tests, const Orbital *__restrict__ orb,
    const double *__restrict__ gtab, double a0, double a1, double a2, int i0, int i1, int i2,
    int gen, LatticeDev lat, Jmat J, double detJ, double *__restrict__ out) {
  __shared__ double r0[RT_NT], r1[RT_NT];
  const RuleTest T = tests[blockIdx.x];
  const int p = T.p, p2 = p * p, p3 = p2 * p;
  const double *gx = gtab + (size_t)p * 2 * RT_PMAX, *gw = gx + RT_PMAX;
  const Orbital o = orb[T.alpha];
  const double av[3] = {a0, a1, a2};
  const int img[3] = {i0, i1, i2};
  double half[3], mid[3];
  for (int k = 0; k < 3; ++k) {
    half[k] = 0.5 * (T.hi[k] - T.lo[k]);
    mid[k] = 0.5 * (T.hi[k] + T.lo[k]);
  }
  double s0 = 0.0, s1 = 0.0;
  for (int k = threadIdx.x; k < p3; k += RT_NT) {
    const int kz = k / p2, ky = (k - kz * p2) / p, kx = k - kz * p2 - ky * p;
    const double pt[3] = {mid[0] + half[0] * gx[kx], mid[1] + half[1] * gx[ky],
                          mid[2] + half[2] * gx[kz]};
    double wt = gw[kx] * gw[ky] * gw[kz] * half[0] * half[1] * half[2];
    double psi, g[3];
    if (gen) {
      double x[3];
      for (int r = 0; r < 3; ++r)
        x[r] = T.x0[r] + J.m[3 * r] * (pt[0] + 1.0) + J.m[3 * r + 1] * (pt[1] + 1.0) +
               J.m[3 * r + 2] * (pt[2] + 1.0);
      enrichment_eval_lat(o, x, lat, psi, g);
      wt *= detJ;
    } else {
      enrichment_eval(o, pt, av, img, psi, g);
    }
    s0 += wt * psi * psi;
    s1 += wt * (g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
  }
  r0[threadIdx.x] = s0;
  r1[threadIdx.x] = s1;
  __syncthreads();
  for (int w = RT_NT / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      r0[threadIdx.x] += r0[threadIdx.x + w];
      r1[threadIdx.x] += r1[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[2 * (size_t)blockIdx.x] = r0[0];
    out[2 * (size_t)blockIdx.x + 1] = r1[0];
  }
}

// Run `tests` on the current device; out[2 t], out[2 t + 1] receive test t's
// integrals.  Blocking; allocates and frees its own device arrays.
static pufe_status device_rule_tests(const Setup &S, const std::vector<RuleTest> &tests,
                                     std::vector<double> &out) {
  out.assign(2 * tests.size(), 0.0);
  if (tests.empty()) return PUFE_OK;
  for (const RuleTest &t : tests)
    if (t.p < 1 || t.p > RT_PMAX || t.alpha < 0 || t.alpha >= (int)S.orb.size())
      return fail(PUFE_EINVAL, "internal: bad adaptive test");
  std::vector<double> gtab((size_t)(RT_PMAX + 1) * 2 * RT_PMAX, 0.0);
  for (int p = 1; p <= RT_PMAX && p < (int)S.gx.size(); ++p)
    for (int i = 0; i < p; ++i) {
      gtab[(size_t)p * 2 * RT_PMAX + i] = S.gx[p][i];
      gtab[(size_t)p * 2 * RT_PMAX + RT_PMAX + i] = S.gw[p][i];
    }
  RuleTest *dt = nullptr;
  Orbital *dorb = nullptr;
  double *dg = nullptr, *dout = nullptr;
  auto release = [&]() {
    if (dt) cudaFree(dt);
    if (dorb) cudaFree(dorb);
    if (dg) cudaFree(dg);
    if (dout) cudaFree(dout);
  };
  auto check = [&](cudaError_t e, const char *what) -> pufe_status {
    if (e == cudaSuccess) return PUFE_OK;
    release();
    return cuda_fail(e, what);
  };
  pufe_status st;
  if ((st = check(cudaMalloc((void **)&dt, tests.size() * sizeof(RuleTest)), "cudaMalloc")))
    return st;
  if ((st = check(cudaMalloc((void **)&dorb, std::max<size_t>(1, S.orb.size()) * sizeof(Orbital)),
                  "cudaMalloc")))
    return st;
  if ((st = check(cudaMalloc((void **)&dg, gtab.size() * sizeof(double)), "cudaMalloc"))) return st;
  if ((st = check(cudaMalloc((void **)&dout, out.size() * sizeof(double)), "cudaMalloc")))
    return st;
  if ((st = check(cudaMemcpy(dt, tests.data(), tests.size() * sizeof(RuleTest),
                             cudaMemcpyHostToDevice), "cudaMemcpy")))
    return st;
  if ((st = check(cudaMemcpy(dorb, S.orb.data(), S.orb.size() * sizeof(Orbital),
                             cudaMemcpyHostToDevice), "cudaMemcpy")))
    return st;
  if ((st = check(cudaMemcpy(dg, gtab.data(), gtab.size() * sizeof(double),
                             cudaMemcpyHostToDevice), "cudaMemcpy")))
    return st;
  Jmat J;
  for (int k = 0; k < 9; ++k) J.m[k] = S.J[k];
  const size_t chunk = (size_t)1 << 30;
  for (size_t t0 = 0; t0 < tests.size(); t0 += chunk) {
    const unsigned nb = (unsigned)std::min(chunk, tests.size() - t0);
    k_rule_tests<<<nb, RT_NT>>>(dt + t0, dorb, dg, S.a[0], S.a[1], S.a[2], S.img[0], S.img[1],
                                S.img[2], S.gen ? 1 : 0, S.lat, J, S.detJ, dout + 2 * t0);
    if ((st = check(cudaGetLastError(), "k_rule_tests launch"))) return st;
  }
  if ((st = check(cudaMemcpy(out.data(), dout, out.size() * sizeof(double),
                             cudaMemcpyDeviceToHost), "cudaMemcpy (adaptive tests)")))
    return st;
  release();
  return PUFE_OK;
}

static void parallel_for(int64_t n, const std::function<void(int64_t)> &fn) {
  unsigned nt = std::max(1u, std::thread::hardware_concurrency());
  nt = (unsigned)std::min<int64_t>(nt, std::max<int64_t>(1, n));
  if (nt <= 1) {
    for (int64_t i = 0; i < n; ++i) fn(i);
    return;
  }
  std::vector<std::thread> th;
  std::atomic<int64_t> next(0);
  for (unsigned t = 0; t < nt; ++t)
    th.emplace_back([&]() {
      for (;;) {
        int64_t i = next.fetch_add(1);
        if (i >= n) break;
        fn(i);
      }
    });
  for (auto &t : th) t.join();
}

template <class T>
static pufe_status upload(T **dst, const std::vector<T> &src) {
  size_t bytes = std::max<size_t>(1, src.size()) * sizeof(T);
  PUFE_CUDA_TRY(cudaMalloc((void **)dst, bytes));
  if (!src.empty()) PUFE_CUDA_TRY(cudaMemcpy(*dst, src.data(), src.size() * sizeof(T),
                                             cudaMemcpyHostToDevice));
  return PUFE_OK;
}

static double factorial(int k) {
  double f = 1.0;
  for (int i = 2; i <= k; ++i) f *= i;
  return f;
}

static pufe_status build(const pufe_cell *cell, const pufe_species *species, int nspecies,
                         const pufe_quad *quad, pufe_ctx *ctx) {
  // ---- validate ----------------------------------------------------------
  if (!cell || !quad) return fail(PUFE_EINVAL, "cell and quad must not be NULL");
  if (cell->natoms < 0 || (cell->natoms > 0 && (!cell->tau || !cell->species)))
    return fail(PUFE_EINVAL, "bad atom arrays");
  if (nspecies < 0 || (nspecies > 0 && !species)) return fail(PUFE_EINVAL, "bad species");
  for (int k = 0; k < 3; ++k) {
    if ((!cell->lattice && !(cell->a[k] > 0.0)) || cell->nel[k] < 1 || cell->nel[k] > 4096)
      return fail(PUFE_EINVAL, "cell edges must be > 0 and nel in [1, 4096]");
  }
  if (quad->mode < PUFE_QUAD_FIXED || quad->mode > PUFE_QUAD_HADAPT)
    return fail(PUFE_EINVAL, "unknown quadrature mode");
  if (quad->mode == PUFE_QUAD_FIXED &&
      (quad->p_far < 1 || quad->p_far > 16 || quad->p_near < 1 || quad->p_near > 16))
    return fail(PUFE_EINVAL, "FIXED rule orders must lie in [1, 16]");
  if (quad->mode == PUFE_QUAD_PADAPT &&
      (quad->p_min < 1 || quad->p_max < quad->p_min || quad->p_max > 16))
    return fail(PUFE_EINVAL, "PADAPT needs 1 <= p_min <= p_max <= 16");
  if (quad->mode == PUFE_QUAD_HADAPT &&
      (quad->max_depth < 0 || quad->max_depth > 4 || quad->p_far < 1 || quad->p_far > 16))
    return fail(PUFE_EINVAL, "HADAPT needs 0 <= max_depth <= 4 and p_far in [1, 16]");
  if (quad->mode != PUFE_QUAD_FIXED && !(quad->tol > 0.0))
    return fail(PUFE_EINVAL, "adaptive tolerance must be > 0");
  if (cell->fe_space != PUFE_FE_LAGRANGE64 && cell->fe_space != PUFE_FE_SERENDIPITY32)
    return fail(PUFE_EINVAL, "unknown FE space");
  const bool ser = cell->fe_space == PUFE_FE_SERENDIPITY32;
  const int nfe_e = ser ? 32 : 64;

  Setup S;
  double rc_max = 0.0;
  if (cell->lattice) {
    // general cell: rows a_d; a[] and h[] hold |a_d| and |a_d| / nel_d
    S.gen = true;
    const double *L = cell->lattice;
    for (int k = 0; k < 9; ++k) S.lat.L[k] = L[k];
    const double det = L[0] * (L[4] * L[8] - L[5] * L[7]) - L[1] * (L[3] * L[8] - L[5] * L[6]) +
                       L[2] * (L[3] * L[7] - L[4] * L[6]);
    double scale = 0.0;
    for (int k = 0; k < 9; ++k) scale = std::max(scale, std::fabs(L[k]));
    if (!(std::fabs(det) > 1e-9 * scale * scale * scale))
      return fail(PUFE_EINVAL, "lattice vectors are (nearly) linearly dependent");
    // L^-T: the cofactor matrix of L over det(L)
    double C[9] = {L[4] * L[8] - L[5] * L[7], L[5] * L[6] - L[3] * L[8], L[3] * L[7] - L[4] * L[6],
                   L[2] * L[7] - L[1] * L[8], L[0] * L[8] - L[2] * L[6], L[1] * L[6] - L[0] * L[7],
                   L[1] * L[5] - L[2] * L[4], L[2] * L[3] - L[0] * L[5], L[0] * L[4] - L[1] * L[3]};
    for (int k = 0; k < 9; ++k) S.lat.Lit[k] = C[k] / det;
    for (int k = 0; k < 3; ++k) {
      S.a[k] = std::sqrt(L[3 * k] * L[3 * k] + L[3 * k + 1] * L[3 * k + 1] + L[3 * k + 2] * L[3 * k + 2]);
      S.nel[k] = cell->nel[k];
      S.h[k] = S.a[k] / cell->nel[k];
    }
    // J = [a_d / 2 nel_d] as columns, J^-T = 2 nel_d (L^-T row d) ... row-wise
    for (int r = 0; r < 3; ++r)
      for (int d = 0; d < 3; ++d) S.J[3 * r + d] = L[3 * d + r] / (2.0 * S.nel[d]);
    for (int r = 0; r < 3; ++r)
      for (int d = 0; d < 3; ++d) S.Jit[3 * r + d] = S.lat.Lit[3 * d + r] * (2.0 * S.nel[d]);
    S.detJ = std::fabs(det) / (8.0 * S.nel[0] * S.nel[1] * S.nel[2]);
  } else {
    for (int k = 0; k < 3; ++k) {
      S.a[k] = cell->a[k];
      S.nel[k] = cell->nel[k];
      S.h[k] = cell->a[k] / cell->nel[k];
    }
  }
  for (int s = 0; s < nspecies; ++s) {
    const pufe_species &sp = species[s];
    if (sp.norb < 0 || (sp.norb > 0 && (!sp.n || !sp.l || !sp.m || !sp.zeta)))
      return fail(PUFE_EINVAL, "bad orbital arrays");
    if (!(sp.r_c > 0.0) || !(sp.r_e >= 0.0)) return fail(PUFE_EINVAL, "need r_c > 0, r_e >= 0");
    for (int o = 0; o < sp.norb; ++o) {
      if (sp.l[o] < 0 || sp.l[o] > 3 || sp.n[o] <= sp.l[o] || sp.n[o] > 8 ||
          sp.m[o] < -sp.l[o] || sp.m[o] > sp.l[o] || !(sp.zeta[o] > 0.0))
        return fail(PUFE_EINVAL, "orbital needs 0<=l<=3, l<n<=8, |m|<=l, zeta>0");
    }
    S.rc_species.push_back(sp.r_c);
    S.re_species.push_back(sp.r_e);
    rc_max = std::max(rc_max, sp.r_c);
  }
  for (int k = 0; k < 3; ++k) S.img[k] = (int)std::ceil(rc_max / S.a[k] + 0.5);
  if (S.gen)   // |s_k| <= r_c |row k of L^-T| for |d| <= r_c, plus the rounding's 1/2
    for (int k = 0; k < 3; ++k) {
      const double nr = std::sqrt(S.lat.Lit[3 * k] * S.lat.Lit[3 * k] +
                                  S.lat.Lit[3 * k + 1] * S.lat.Lit[3 * k + 1] +
                                  S.lat.Lit[3 * k + 2] * S.lat.Lit[3 * k + 2]);
      S.img[k] = (int)std::ceil(rc_max * nr + 0.5);
    }
  for (int k = 0; k < 3; ++k) S.lat.img[k] = S.img[k];
  for (int ia = 0; ia < cell->natoms; ++ia) {
    int s = cell->species[ia];
    if (s < 0 || s >= nspecies) return fail(PUFE_EINVAL, "atom species out of range");
    S.tau.push_back({cell->tau[3 * ia], cell->tau[3 * ia + 1], cell->tau[3 * ia + 2]});
    S.atom_species.push_back(s);
    const pufe_species &sp = species[s];
    for (int o = 0; o < sp.norb; ++o) {
      Orbital ob;
      for (int k = 0; k < 3; ++k) ob.tau[k] = cell->tau[3 * ia + k];
      ob.n = sp.n[o];
      ob.l = sp.l[o];
      ob.m = sp.m[o];
      ob.zeta = sp.zeta[o];
      ob.rc = sp.r_c;
      ob.norm = std::pow(2.0 * ob.zeta, ob.n + 0.5) / std::sqrt(factorial(2 * ob.n));
      ob.pad = 0;
      S.orb.push_back(ob);
      S.orb_atom.push_back(ia);
    }
  }
  S.gx.resize(19);
  S.gw.resize(19);
  for (int p = 1; p <= 18; ++p) gauss_legendre(p, S.gx[p], S.gw[p]);  // PADAPT reads p_max + 2

  const int nx = S.nel[0], ny = S.nel[1], nz = S.nel[2];
  const int64_t nelem = (int64_t)nx * ny * nz;
  const int64_t nv = nelem;
  const int mx = 3 * nx, my = 3 * ny, mz = 3 * nz;
  // FE DOFs: the nodes of the periodic (3 nx)(3 ny)(3 nz) grid; for the
  // serendipity space only those with at most one coordinate off the vertex
  // planes, numbered compactly in grid order (gmap: grid index -> DOF)
  std::vector<int32_t> gmap;
  int64_t n_fe = (int64_t)mx * my * mz;
  if (ser) {
    gmap.assign((size_t)n_fe, -1);
    int64_t k = 0;
    for (int64_t g = 0; g < (int64_t)mx * my * mz; ++g) {
      const int64_t gx = g % mx, gy = (g / mx) % my, gz = g / ((int64_t)mx * my);
      if ((gx % 3 != 0) + (gy % 3 != 0) + (gz % 3 != 0) <= 1) gmap[g] = (int32_t)k++;
    }
    n_fe = k;
  }
  const int natoms = cell->natoms;

  // the element's box: physical for orthorhombic cells, the reference cube
  // for general ones (mapped by x0(e) + J (xi + 1))
  auto elem_box = [&](int64_t e) {
    int ex = (int)(e % nx), ey = (int)((e / nx) % ny), ez = (int)(e / ((int64_t)nx * ny));
    Box b;
    int idx[3] = {ex, ey, ez};
    for (int k = 0; k < 3; ++k) {
      b.lo[k] = S.gen ? -1.0 : idx[k] * S.h[k];
      b.hi[k] = S.gen ? 1.0 : b.lo[k] + S.h[k];
    }
    return b;
  };
  auto origin = [&](int64_t e, double x0[3]) {
    int idx[3] = {(int)(e % nx), (int)((e / nx) % ny), (int)(e / ((int64_t)nx * ny))};
    elem_origin(S, idx, x0);
  };
  auto elem_vertex = [&](int64_t e, int lv) -> int64_t {
    int ex = (int)(e % nx), ey = (int)((e / nx) % ny), ez = (int)(e / ((int64_t)nx * ny));
    int a = lv & 1, b = (lv >> 1) & 1, c = (lv >> 2) & 1;
    return ((ex + a) % nx) + (int64_t)nx * (((ey + b) % ny) + (int64_t)ny * ((ez + c) % nz));
  };

  // ---- element / atom proximity ------------------------------------------
  std::vector<uint8_t> near((size_t)nelem * std::max(1, natoms), 0);
  parallel_for(nelem, [&](int64_t e) {
    Box b = elem_box(e);
    double x0[3], M[9];
    if (S.gen) {
      origin(e, x0);
      for (int k = 0; k < 9; ++k) M[k] = 2.0 * S.J[k];
    }
    for (int ia = 0; ia < natoms; ++ia) {
      double d;
      if (S.gen) {   // images within the half-widths, one more for the rounding
        d = 1e300;
        const int R0 = S.img[0] + 1, R1 = S.img[1] + 1, R2 = S.img[2] + 1;
        for (int i = -R0; i <= R0; ++i)
          for (int j = -R1; j <= R1; ++j)
            for (int k = -R2; k <= R2; ++k) {
              double P[3];
              for (int r = 0; r < 3; ++r)
                P[r] = S.tau[ia][r] + i * S.lat.L[r] + j * S.lat.L[3 + r] + k * S.lat.L[6 + r];
              d = std::min(d, parallelepiped_point_dist(x0, M, P));
            }
      } else {
        d = atom_box_dist(S, S.tau[ia].data(), b);
      }
      near[(size_t)e * natoms + ia] = d < S.rc_species[S.atom_species[ia]] ? 1 : 0;
    }
  });

  // ---- enriched vertices per atom (minimum image distance <= r_e) --------
  std::vector<std::vector<int64_t>> enr_verts(natoms);
  for (int ia = 0; ia < natoms; ++ia) {
    double re = S.re_species[S.atom_species[ia]];
    for (int64_t v = 0; v < nv; ++v) {
      int vx = (int)(v % nx), vy = (int)((v / nx) % ny), vz = (int)(v / ((int64_t)nx * ny));
      int vi[3] = {vx, vy, vz};
      double s = 0.0;
      if (S.gen) {   // lattice-coordinate rounding, then the neighbouring images
        double x[3], d[3], f[3];
        elem_origin(S, vi, x);
        for (int k = 0; k < 3; ++k) d[k] = x[k] - S.tau[ia][k];
        for (int k = 0; k < 3; ++k) {
          f[k] = S.lat.Lit[3 * k] * d[0] + S.lat.Lit[3 * k + 1] * d[1] + S.lat.Lit[3 * k + 2] * d[2];
          f[k] -= std::nearbyint(f[k]);
        }
        s = 1e300;
        for (int i = -1; i <= 1; ++i)
          for (int j = -1; j <= 1; ++j)
            for (int k = -1; k <= 1; ++k) {
              double t = 0.0;
              for (int r = 0; r < 3; ++r) {
                const double c = (f[0] + i) * S.lat.L[r] + (f[1] + j) * S.lat.L[3 + r] +
                                 (f[2] + k) * S.lat.L[6 + r];
                t += c * c;
              }
              s = std::min(s, t);
            }
      } else {
        for (int k = 0; k < 3; ++k) {
          double d = vi[k] * S.h[k] - S.tau[ia][k];
          d -= S.a[k] * std::nearbyint(d / S.a[k]);
          s += d * d;
        }
      }
      if (std::sqrt(s) <= re + 1e-12) enr_verts[ia].push_back(v);
    }
  }

  // ---- enrichment DOFs and element columns --------------------------------
  std::vector<std::vector<std::pair<int64_t, int>>> vert_elems(nv);  // (e, lv)
  for (int64_t e = 0; e < nelem; ++e)
    for (int lv = 0; lv < 8; ++lv) vert_elems[elem_vertex(e, lv)].push_back({e, lv});
  struct Col {
    int64_t dof;
    int lv;
    int alpha;
  };
  std::vector<std::vector<Col>> cols(nelem);
  int64_t dof = n_fe;
  for (size_t k = 0; k < S.orb.size(); ++k) {
    int ia = S.orb_atom[k];
    for (int64_t v : enr_verts[ia]) {
      bool any = false;
      for (auto &el : vert_elems[v]) {
        if (near[(size_t)el.first * natoms + ia]) {
          cols[el.first].push_back({dof, el.second, (int)k});
          any = true;
        }
      }
      if (any) ++dof;
    }
  }
  const int64_t n_dof = dof;
  if (n_dof > INT32_MAX) return fail(PUFE_EINVAL, "too many DOFs for int32 column indices");
  for (auto &c : cols)
    std::sort(c.begin(), c.end(), [](const Col &x, const Col &y) {
      return x.dof != y.dof ? x.dof < y.dof : x.lv < y.lv;
    });

  // per-element alpha lists
  std::vector<std::vector<int>> ealpha(nelem);
  for (int64_t e = 0; e < nelem; ++e) {
    for (auto &c : cols[e]) ealpha[e].push_back(c.alpha);
    std::sort(ealpha[e].begin(), ealpha[e].end());
    ealpha[e].erase(std::unique(ealpha[e].begin(), ealpha[e].end()), ealpha[e].end());
  }

  // ---- quadrature rules ----------------------------------------------------
  std::vector<std::vector<RulePart>> rule(nelem);
  if (quad->device_tests && quad->mode != PUFE_QUAD_FIXED) {
    // the integrals of the adaptive tests on the GPU, one launch per order
    // set (PADAPT) or per subdivision level (HADAPT); same decisions, points
    // and order as the host construction below
    int ndev0 = 0;
    if (cudaGetDeviceCount(&ndev0) != cudaSuccess || ndev0 == 0) {
      cudaGetLastError();
      return fail(PUFE_ECUDA, "quad.device_tests needs a CUDA device");
    }
    auto make_test = [&](int64_t e, const Box &b, int alpha, int p) {
      RuleTest t;
      for (int k = 0; k < 3; ++k) {
        t.lo[k] = b.lo[k];
        t.hi[k] = b.hi[k];
        t.x0[k] = 0.0;
      }
      if (S.gen) origin(e, t.x0);
      t.alpha = alpha;
      t.p = p;
      return t;
    };
    std::vector<double> out;
    pufe_status st0;
    if (quad->mode == PUFE_QUAD_PADAPT) {
      const int p0 = quad->p_min, p1 = quad->p_max + 2;
      std::vector<RuleTest> tests;
      std::vector<int64_t> first(nelem + 1, 0);
      for (int64_t e = 0; e < nelem; ++e) {
        first[e] = (int64_t)tests.size();
        const Box b = elem_box(e);
        for (int p = p0; p <= p1; ++p)
          for (int al : ealpha[e]) tests.push_back(make_test(e, b, al, p));
      }
      first[nelem] = (int64_t)tests.size();
      if ((st0 = device_rule_tests(S, tests, out)) != PUFE_OK) return st0;
      for (int64_t e = 0; e < nelem; ++e) {
        const Box b = elem_box(e);
        const int64_t A = (int64_t)ealpha[e].size();
        if (A == 0) {
          rule[e].push_back({b, quad->p_min});
          continue;
        }
        // I_p of integrand i (2 per enrichment) of element e
        auto I = [&](int p, int64_t i) { return out[2 * (first[e] + (p - p0) * A) + i]; };
        int chosen = quad->p_max;
        for (int p = quad->p_min; p <= quad->p_max; ++p) {
          bool ok = true;
          for (int64_t i = 0; i < 2 * A; ++i) ok = ok && (std::fabs(I(p, i) - I(p + 2, i)) < quad->tol);
          if (ok) {
            chosen = p;
            break;
          }
        }
        rule[e].push_back({b, chosen});
      }
    } else {
      // HADAPT: a tree per element, tested level by level; leaves emitted
      // depth first in the host's child order a + 2 b + 4 c
      struct Node {
        int64_t e;
        Box b;
        std::vector<int> al;
        int depth, child0;
      };
      std::vector<Node> nodes;
      std::vector<int64_t> root(nelem, -1);
      std::vector<int64_t> level;
      for (int64_t e = 0; e < nelem; ++e) {
        if (ealpha[e].empty()) continue;
        root[e] = (int64_t)nodes.size();
        level.push_back(root[e]);
        nodes.push_back(Node{e, elem_box(e), ealpha[e], 0, -1});
      }
      while (!level.empty()) {
        std::vector<RuleTest> tests;
        std::vector<int64_t> first;
        for (int64_t id : level) {
          first.push_back((int64_t)tests.size());
          for (int al : nodes[id].al) {
            tests.push_back(make_test(nodes[id].e, nodes[id].b, al, 5));
            tests.push_back(make_test(nodes[id].e, nodes[id].b, al, 8));
          }
        }
        if ((st0 = device_rule_tests(S, tests, out)) != PUFE_OK) return st0;
        std::vector<int64_t> next;
        for (size_t j = 0; j < level.size(); ++j) {
          const int64_t id = level[j];
          std::vector<int> failing;
          for (size_t ia = 0; ia < nodes[id].al.size(); ++ia) {
            const double *i5 = &out[2 * (first[j] + 2 * (int64_t)ia)], *i8 = i5 + 2;
            if (std::fabs(i5[0] - i8[0]) >= quad->tol || std::fabs(i5[1] - i8[1]) >= quad->tol)
              failing.push_back(nodes[id].al[ia]);
          }
          if (failing.empty() || nodes[id].depth >= quad->max_depth) continue;
          const Box pb = nodes[id].b;
          double mid[3];
          for (int k = 0; k < 3; ++k) mid[k] = 0.5 * (pb.lo[k] + pb.hi[k]);
          nodes[id].child0 = (int)nodes.size();
          const int64_t e = nodes[id].e;
          const int depth = nodes[id].depth + 1;
          for (int c = 0; c < 2; ++c)
            for (int bb = 0; bb < 2; ++bb)
              for (int a = 0; a < 2; ++a) {
                const int off[3] = {a, bb, c};
                Box ch;
                for (int k = 0; k < 3; ++k) {
                  ch.lo[k] = off[k] == 0 ? pb.lo[k] : mid[k];
                  ch.hi[k] = off[k] == 0 ? mid[k] : pb.hi[k];
                }
                next.push_back((int64_t)nodes.size());
                nodes.push_back(Node{e, ch, failing, depth, -1});
              }
        }
        level.swap(next);
      }
      for (int64_t e = 0; e < nelem; ++e) {
        if (root[e] < 0) {
          rule[e].push_back({elem_box(e), quad->p_far});
          continue;
        }
        std::function<void(int64_t)> emit = [&](int64_t id) {
          if (nodes[id].child0 < 0) {
            rule[e].push_back({nodes[id].b, 8});
            return;
          }
          for (int c = 0; c < 8; ++c) emit(nodes[id].child0 + c);
        };
        emit(root[e]);
      }
    }
  } else
  parallel_for(nelem, [&](int64_t e) {
    Box b = elem_box(e);
    double x0v[3];
    if (S.gen) origin(e, x0v);
    const double *x0 = S.gen ? x0v : nullptr;
    std::vector<RulePart> &parts = rule[e];
    if (quad->mode == PUFE_QUAD_FIXED) {
      bool nr = false;
      for (int ia = 0; ia < natoms; ++ia) nr = nr || near[(size_t)e * natoms + ia];
      parts.push_back({b, nr ? quad->p_near : quad->p_far});
    } else if (quad->mode == PUFE_QUAD_PADAPT) {
      const std::vector<int> &al = ealpha[e];
      if (al.empty()) {
        parts.push_back({b, quad->p_min});
        return;
      }
      std::vector<std::vector<double>> I(quad->p_max + 3);
      auto get = [&](int p) -> const std::vector<double> & {
        if (I[p].empty()) box_integrals(S, al, b, p, I[p], x0);
        return I[p];
      };
      int chosen = quad->p_max;
      for (int p = quad->p_min; p <= quad->p_max; ++p) {
        const std::vector<double> &a1 = get(p), &a2 = get(p + 2);
        bool ok = true;
        for (size_t i = 0; i < a1.size(); ++i) ok = ok && (std::fabs(a1[i] - a2[i]) < quad->tol);
        if (ok) {
          chosen = p;
          break;
        }
      }
      parts.push_back({b, chosen});
    } else {
      if (ealpha[e].empty()) {
        parts.push_back({b, quad->p_far});
        return;
      }
      hadapt(S, ealpha[e], b, 0, *quad, parts, x0);
    }
  });
  std::vector<int64_t> qoff(nelem + 1, 0);
  for (int64_t e = 0; e < nelem; ++e) {
    int64_t q = 0;
    for (auto &pt : rule[e]) q += (int64_t)pt.p * pt.p * pt.p;
    qoff[e + 1] = qoff[e] + q;
  }
  const int64_t nq = qoff[nelem];
  std::vector<double> X(3 * nq), Wt(nq), XI(3 * nq);
  parallel_for(nelem, [&](int64_t e) {
    Box eb = elem_box(e);
    double x0[3] = {0, 0, 0};
    if (S.gen) origin(e, x0);
    int64_t q = qoff[e];
    for (auto &pt : rule[e]) {
      const std::vector<double> &gx = S.gx[pt.p], &gw = S.gw[pt.p];
      double half[3], mid[3];
      for (int k = 0; k < 3; ++k) {
        half[k] = 0.5 * (pt.box.hi[k] - pt.box.lo[k]);
        mid[k] = 0.5 * (pt.box.hi[k] + pt.box.lo[k]);
      }
      for (int kz = 0; kz < pt.p; ++kz)
        for (int ky = 0; ky < pt.p; ++ky)
          for (int kx = 0; kx < pt.p; ++kx, ++q) {
            int kk[3] = {kx, ky, kz};
            if (S.gen) {   // reference point of the sub-box, mapped by the element
              for (int d = 0; d < 3; ++d) XI[3 * q + d] = mid[d] + half[d] * gx[kk[d]];
              for (int r = 0; r < 3; ++r)
                X[3 * q + r] = x0[r] + S.J[3 * r] * (XI[3 * q] + 1.0) +
                               S.J[3 * r + 1] * (XI[3 * q + 1] + 1.0) +
                               S.J[3 * r + 2] * (XI[3 * q + 2] + 1.0);
              Wt[q] = gw[kx] * gw[ky] * gw[kz] * half[0] * half[1] * half[2] * S.detJ;
            } else {
              for (int d = 0; d < 3; ++d) {
                X[3 * q + d] = mid[d] + half[d] * gx[kk[d]];
                XI[3 * q + d] = 2.0 * (X[3 * q + d] - eb.lo[d]) / S.h[d] - 1.0;
              }
              Wt[q] = gw[kx] * gw[ky] * gw[kz] * half[0] * half[1] * half[2];
            }
          }
    }
  });

  // ---- element DOF lists, column descriptors, alpha slots ------------------
  std::vector<int64_t> doff(nelem + 1, 0), toff(nelem + 1, 0);
  std::vector<int32_t> aoff(nelem + 1, 0);
  std::vector<int32_t> n_e(nelem), q_e(nelem);
  for (int64_t e = 0; e < nelem; ++e) {
    n_e[e] = nfe_e + (int32_t)cols[e].size();
    q_e[e] = (int32_t)(qoff[e + 1] - qoff[e]);
    doff[e + 1] = doff[e] + n_e[e];
    aoff[e + 1] = aoff[e] + (int32_t)ealpha[e].size();
    toff[e + 1] = toff[e] + (int64_t)q_e[e] * (int64_t)ealpha[e].size();
  }
  // FP32 path: points padded to multiples of 8, chunk-blocked table offsets
  std::vector<int64_t> qpoff(nelem + 1, 0), toff32(nelem + 1, 0);
  for (int64_t e = 0; e < nelem; ++e) {
    const int64_t qp = ((int64_t)q_e[e] + 7) / 8 * 8;
    qpoff[e + 1] = qpoff[e] + qp;
    toff32[e + 1] = toff32[e] + qp * (int64_t)ealpha[e].size();
  }
  std::vector<float4> qdat(qpoff[nelem]);
  std::vector<float> ptab(32 * qpoff[nelem], 0.0f);
  std::vector<float> eorig(8 * aoff[nelem], 0.0f);
  std::vector<int32_t> dofs(doff[nelem]), ecol(doff[nelem] - nfe_e * nelem), alist(aoff[nelem]);
  // lattice shift of every element column's node or vertex (bit d: one cell
  // along axis d), for the Bloch phases at k != 0
  std::vector<uint8_t> eshift(doff[nelem]);
  int64_t ecpos = 0;
  for (int64_t e = 0; e < nelem; ++e) {
    int ex = (int)(e % nx), ey = (int)((e / nx) % ny), ez = (int)(e / ((int64_t)nx * ny));
    int32_t *d = &dofs[doff[e]];
    for (int j = 0; j < nfe_e; ++j) {   // FE columns: local node a + 4 b + 16 c
      const int loc = ser ? ser_local(j) : j;
      const int a = loc & 3, b = (loc >> 2) & 3, c = loc >> 4;
      const int64_t gx = (3 * ex + a) % mx, gy = (3 * ey + b) % my, gz = (3 * ez + c) % mz;
      const int64_t g = gx + mx * (gy + (int64_t)my * gz);
      d[j] = ser ? gmap[g] : (int32_t)g;
      eshift[doff[e] + j] = (uint8_t)((3 * ex + a >= mx ? 1 : 0) | (3 * ey + b >= my ? 2 : 0) |
                                      (3 * ez + c >= mz ? 4 : 0));
    }
    for (size_t k = 0; k < ealpha[e].size(); ++k) {
      alist[aoff[e] + k] = ealpha[e][k];
      // element origin minus the nearest image of the atom, split hi + lo
      const Orbital &o = S.orb[ealpha[e][k]];
      const Box b = elem_box(e);
      float *dst = &eorig[8 * (aoff[e] + k)];
      for (int d = 0; d < 3 && !S.gen; ++d) {   // (the FP32 path takes orthorhombic cells)
        double v = b.lo[d] - o.tau[d];
        v -= S.a[d] * std::floor(v / S.a[d] + 0.5);
        const float hi = (float)v;
        dst[d] = hi;
        dst[3 + d] = (float)(v - (double)hi);
      }
    }
    for (int64_t q = 0; q < qpoff[e + 1] - qpoff[e]; ++q) {
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (q < q_e[e]) {
        const int64_t g = qoff[e] + q;
        v = make_float4((float)XI[3 * g], (float)XI[3 * g + 1], (float)XI[3 * g + 2], (float)Wt[g]);
        float *pt = &ptab[32 * (qpoff[e] + q)];
        for (int d = 0; d < 3; ++d) {
          double L[4], dL[4];
          lagrange3(XI[3 * g + d], L, dL);
          for (int c = 0; c < 4; ++c) {
            pt[4 * d + c] = (float)L[c];
            pt[12 + 4 * d + c] = (float)(dL[c] * 2.0 / S.h[d]);
          }
          pt[24 + d] = (float)XI[3 * g + d];
        }
        pt[27] = (float)std::sqrt(0.5 * Wt[g]);
        pt[28] = (float)std::sqrt(Wt[g]);
      }
      qdat[qpoff[e] + q] = v;
    }
    for (size_t j = 0; j < cols[e].size(); ++j) {
      d[nfe_e + j] = (int32_t)cols[e][j].dof;
      int slot = (int)(std::lower_bound(ealpha[e].begin(), ealpha[e].end(), cols[e][j].alpha) -
                       ealpha[e].begin());
      ecol[ecpos++] = (slot << 3) | cols[e][j].lv;
      const int lv = cols[e][j].lv;
      eshift[doff[e] + nfe_e + j] = (uint8_t)((ex + (lv & 1) >= nx ? 1 : 0) |
                                           (ey + ((lv >> 1) & 1) >= ny ? 2 : 0) |
                                           (ez + (lv >> 2) >= nz ? 4 : 0));
    }
  }

  // ---- CSR pattern (union of element blocks) ------------------------------
  std::vector<std::vector<int32_t>> rows(n_dof);
  {
    // row lists built per element, then sorted/uniqued per row
    for (int64_t e = 0; e < nelem; ++e) {
      const int32_t *d = &dofs[doff[e]];
      int n = n_e[e];
      for (int i = 0; i < n; ++i) {
        std::vector<int32_t> &r = rows[d[i]];
        r.insert(r.end(), d, d + n);
      }
    }
    parallel_for(n_dof, [&](int64_t r) {
      std::vector<int32_t> &v = rows[r];
      std::sort(v.begin(), v.end());
      v.erase(std::unique(v.begin(), v.end()), v.end());
      v.shrink_to_fit();
    });
  }
  std::vector<int64_t> rowptr(n_dof + 1, 0);
  for (int64_t r = 0; r < n_dof; ++r) rowptr[r + 1] = rowptr[r] + (int64_t)rows[r].size();
  const int64_t nnz = rowptr[n_dof];
  if (nnz > INT32_MAX) return fail(PUFE_EINVAL, "nnz exceeds int32 scatter slots");
  std::vector<int32_t> colv(nnz);
  parallel_for(n_dof, [&](int64_t r) {
    std::copy(rows[r].begin(), rows[r].end(), colv.begin() + rowptr[r]);
  });
  rows.clear();
  rows.shrink_to_fit();

  std::vector<int64_t> soff(nelem + 1, 0);
  for (int64_t e = 0; e < nelem; ++e) soff[e + 1] = soff[e] + (int64_t)n_e[e] * n_e[e];
  std::vector<int32_t> smap(soff[nelem]);
  parallel_for(nelem, [&](int64_t e) {
    const int32_t *d = &dofs[doff[e]];
    int n = n_e[e];
    int32_t *m = &smap[soff[e]];
    for (int i = 0; i < n; ++i) {
      const int32_t *b = colv.data() + rowptr[d[i]], *en = colv.data() + rowptr[d[i] + 1];
      for (int j = 0; j < n; ++j) {
        const int32_t *f = std::lower_bound(b, en, d[j]);
        m[(int64_t)i * n + j] = (int32_t)(f - colv.data());
      }
    }
  });

  // ---- work order: elements with n_e > 128 first (they take the 256-row
  // tile), then by decreasing cost n_e^2 Q_e (largest first balances the
  // per-element launches and the persistent round-robin schedule) -----------
  std::vector<int32_t> order(nelem);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) {
    const bool bx = n_e[x] > 128, by = n_e[y] > 128;
    if (bx != by) return bx;
    int64_t cx = (int64_t)n_e[x] * n_e[x] * q_e[x], cy = (int64_t)n_e[y] * n_e[y] * q_e[y];
    return cx > cy;
  });
  int n_big = 0;
  for (int64_t e = 0; e < nelem; ++e) n_big += n_e[e] > 128 ? 1 : 0;

  // ---- constant FE-FE blocks (exact for rules with >= 4 points per axis) -----
  // 1D cubic Lagrange mass/stiffness on [-1, 1] by the 4-point Gauss rule,
  // which is exact for their degree-6 integrands.
  int min_p = 1 << 30;
  for (auto &parts : rule)
    for (auto &pt : parts) min_p = std::min(min_p, pt.p);
  // (the exact FE-FE constants serve the mixed path, which takes the tricubic space)
  const bool fe_exact = min_p >= 4 && !ser;
  std::vector<double> TF, SF, S0;
  if (fe_exact) {
    double M1[4][4] = {{0}}, K1[4][4] = {{0}}, D1[4][4] = {{0}};   // D1[a][b] = int L'_a L_b
    for (int g = 0; g < 4; ++g) {
      double L[4], dL[4];
      lagrange3(S.gx[4][g], L, dL);
      for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) {
          M1[a][b] += S.gw[4][g] * L[a] * L[b];
          K1[a][b] += S.gw[4][g] * dL[a] * dL[b];
          D1[a][b] += S.gw[4][g] * dL[a] * L[b];
        }
    }
    SF.assign(64 * 64, 0.0);
    TF.assign(64 * 64, 0.0);
    if (!S.gen) {
      const double J = 0.125 * S.h[0] * S.h[1] * S.h[2];
      const double s2[3] = {4.0 / (S.h[0] * S.h[0]), 4.0 / (S.h[1] * S.h[1]), 4.0 / (S.h[2] * S.h[2])};
      for (int i = 0; i < 64; ++i)
        for (int j = 0; j < 64; ++j) {
          const int ia[3] = {i & 3, (i >> 2) & 3, i >> 4}, ja[3] = {j & 3, (j >> 2) & 3, j >> 4};
          const double mx = M1[ia[0]][ja[0]], my = M1[ia[1]][ja[1]], mz = M1[ia[2]][ja[2]];
          SF[i * 64 + j] = J * mx * my * mz;
          TF[i * 64 + j] = 0.5 * J * (s2[0] * K1[ia[0]][ja[0]] * my * mz +
                                      s2[1] * mx * K1[ia[1]][ja[1]] * mz +
                                      s2[2] * mx * my * K1[ia[2]][ja[2]]);
        }
    } else {
      // grad phi_i . grad phi_j = sum_kl G_kl d_k phi_i d_l phi_j with the
      // reference metric G = J^-1 J^-T; each term is a product of 1D
      // integrals: M1 on the other axes, K1 when k = l, D1 (and its
      // transpose) on axes k and l when k != l
      double G[3][3];
      for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) {
          G[k][l] = 0.0;
          for (int r = 0; r < 3; ++r) G[k][l] += S.Jit[3 * r + k] * S.Jit[3 * r + l];
        }
      for (int i = 0; i < 64; ++i)
        for (int j = 0; j < 64; ++j) {
          const int ia[3] = {i & 3, (i >> 2) & 3, i >> 4}, ja[3] = {j & 3, (j >> 2) & 3, j >> 4};
          double m = 1.0;
          for (int d = 0; d < 3; ++d) m *= M1[ia[d]][ja[d]];
          SF[i * 64 + j] = S.detJ * m;
          double t = 0.0;
          for (int k = 0; k < 3; ++k)
            for (int l = 0; l < 3; ++l) {
              double f = G[k][l];
              for (int d = 0; d < 3; ++d) {
                if (d == k && d == l) f *= K1[ia[d]][ja[d]];
                else if (d == k) f *= D1[ia[d]][ja[d]];
                else if (d == l) f *= D1[ja[d]][ia[d]];
                else f *= M1[ia[d]][ja[d]];
              }
              t += f;
            }
          TF[i * 64 + j] = 0.5 * S.detJ * t;
        }
    }
    // the overlap constants summed over the elements through the scatter map
    S0.assign(nnz, 0.0);
    for (int64_t e = 0; e < nelem; ++e) {
      const int n = n_e[e];
      const int32_t *m = &smap[soff[e]];
      for (int i = 0; i < 64; ++i)
        for (int j = 0; j < 64; ++j) S0[m[(int64_t)i * n + j]] += SF[i * 64 + j];
    }
  }

  // ---- fill the context and upload ----------------------------------------
  for (int k = 0; k < 3; ++k) {
    ctx->a[k] = S.a[k];
    ctx->h[k] = S.h[k];
    ctx->nel[k] = S.nel[k];
    ctx->images[k] = S.img[k];
  }
  ctx->general = S.gen;
  ctx->ser = ser;
  ctx->nfe_e = nfe_e;
  for (int k = 0; k < 9; ++k) {
    ctx->lat[k] = S.gen ? S.lat.L[k] : 0.0;
    ctx->Jit[k] = S.gen ? S.Jit[k] : 0.0;
  }
  ctx->nelem = nelem;
  ctx->nq = nq;
  ctx->n_dof = n_dof;
  ctx->n_fe = n_fe;
  ctx->nnz = nnz;
  ctx->n_alpha = (int64_t)S.orb.size();
  ctx->psi_len = 4 * toff[nelem];
  ctx->nq_pad = qpoff[nelem];
  ctx->big_pad_end = 0;
  for (int64_t e = 0; e < nelem; ++e)
    if (n_e[e] > 128) ctx->big_pad_end = std::max<int64_t>(ctx->big_pad_end, qpoff[e + 1]);
  ctx->psi32_len = 4 * toff32[nelem];
  ctx->smap_len = soff[nelem];
  ctx->dof_len = doff[nelem];
  ctx->max_basis = *std::max_element(n_e.begin(), n_e.end());
  ctx->max_q = *std::max_element(q_e.begin(), q_e.end());
  ctx->fe_exact = fe_exact;
  ctx->n_big = n_big;
  // (sub)cell structure of every element's rule
  std::vector<int32_t> partoff(nelem + 1, 0), part_p, part_q;
  int max_part_p = 0;
  for (int64_t e = 0; e < nelem; ++e) {
    int32_t qrel = 0;
    for (auto &pt : rule[e]) {
      part_p.push_back(pt.p);
      part_q.push_back(qrel);
      qrel += pt.p * pt.p * pt.p;
      max_part_p = std::max(max_part_p, pt.p);
    }
    partoff[e + 1] = (int32_t)part_p.size();
  }
  ctx->max_part_p = max_part_p;
  ctx->max_alpha = 0;
  for (auto &v : ealpha) ctx->max_alpha = std::max(ctx->max_alpha, (int)v.size());
  // shared-memory stage of the strip kernel: the largest (sub)cell's Psi
  // rows (odd pitch), points and V among enriched elements with
  // n_e <= 128, capped at 10240 floats (larger cells read global memory)
  ctx->strip_stage = 0;
  ctx->strip_pmask = 0;
  ctx->strip_npair_max = 0;
  ctx->adj_sf_floats = 0;
  ctx->adj_sf_all = true;
  ctx->part_p_host.assign(nelem, {});
  for (int64_t e = 0; e < nelem; ++e)
    for (auto &pt : rule[e]) ctx->part_p_host[e].push_back(pt.p);
  ctx->eeform_host.assign(nelem, 0);
  ctx->n_slot.assign(nelem, 0);
  for (int64_t e = 0; e < nelem; ++e) ctx->n_slot[e] = (int32_t)ealpha[e].size();
  ctx->see_stage.assign(nelem, 0);
  for (int64_t e = 0; e < nelem; ++e) {
    if (n_e[e] <= 64) continue;
    int p3max = 0;
    for (int32_t j = partoff[e]; j < partoff[e + 1]; ++j)
      p3max = std::max(p3max, (int)(part_p[j] * part_p[j] * part_p[j]));
    ctx->see_stage[e] = (int32_t)ealpha[e].size() * p3max;
  }
  for (int64_t e = 0; e < nelem; ++e) {
    if (n_e[e] <= 64 || n_e[e] > 128) continue;
    const int A = (int)ealpha[e].size();
    if (A <= 8) ctx->strip_npair_max = std::max(ctx->strip_npair_max, A * (A + 1) / 2);
    int pmax = 0;
    for (int32_t j = partoff[e]; j < partoff[e + 1]; ++j) pmax = std::max(pmax, (int)part_p[j]);
    if (adjoint_sf_fits(A, pmax))
      ctx->adj_sf_floats = std::max(ctx->adj_sf_floats,
                                    A * 512 + A * (A + 1) / 2 * 27 + A * pmax * pmax * pmax);
    else
      ctx->adj_sf_all = false;
    for (int32_t j = partoff[e]; j < partoff[e + 1]; ++j) {
      if (part_p[j] < 32) ctx->strip_pmask |= 1u << part_p[j];
      const int p3 = part_p[j] * part_p[j] * part_p[j];
      const int need = ((A * 4 * (p3 | 1) + 3) & ~3) + 5 * p3;
      if (need <= 10240) ctx->strip_stage = std::max(ctx->strip_stage, need);
    }
  }

  // Device copies: made here when a CUDA device is present.  Without one the
  // context keeps its host-side description only (getters work, compute
  // calls report PUFE_ESTATE).
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    ctx->on_device = false;
  } else {
    PUFE_CUDA_TRY(cudaGetDevice(&ctx->device));
    ctx->on_device = true;
  }
  // ---- FP64 work list ---------------------------------------------------------
  // The FP64 assembly and adjoint take one CTA per work item.  An element
  // whose cost Q_e * npad_e^2 exceeds the mean cost of a CTA slot (two per
  // SM) is cut into point ranges: multiples of 8 points (the kernels' chunk),
  // at least 64 points each.  The ranges' partial element matrices meet in
  // the atomic scatter; the adjoint's ranges write disjoint points.  Items
  // run largest first.  No list (one CTA per element, in `order`) when no
  // element is cut.
  std::vector<int32_t> wsplit;
  {
    int nsm = 152;
    if (ctx->on_device) {
      int v = 0;
      if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, ctx->device) == cudaSuccess &&
          v > 0)
        nsm = v;
    }
    auto cost = [&](int64_t e, int64_t npts) {
      const int64_t np = (n_e[e] + 3) & ~3;
      return (double)npts * (double)(np * np);
    };
    double total = 0.0;
    for (int64_t e = 0; e < nelem; ++e) total += cost(e, q_e[e]);
    const double cmax = std::max(1.0, total / (2.0 * nsm));
    struct Item {
      int32_t e, qa, qb;
      double c;
    };
    std::vector<Item> items;
    bool cut = false;
    for (int64_t e = 0; e < nelem; ++e) {
      const int32_t Q = q_e[e];
      int m = (int)std::min<double>(std::ceil(cost(e, Q) / cmax), 1e6);
      m = std::max(1, std::min(m, Q / 64));
      if (m > 1) cut = true;
      int32_t prev = 0;
      for (int j = 1; j <= m; ++j) {
        const int32_t b = (j == m) ? Q : (int32_t)(((int64_t)j * Q / m) & ~(int64_t)7);
        items.push_back(Item{(int32_t)e, prev, b, cost(e, b - prev)});
        prev = b;
      }
    }
    if (cut) {
      std::stable_sort(items.begin(), items.end(),
                       [](const Item &x, const Item &y) { return x.c > y.c; });
      // every element's points covered exactly once, in ranges inside [0, Q_e)
      std::vector<int64_t> covered(nelem, 0);
      for (const Item &it : items) {
        if (it.qa < 0 || it.qb <= it.qa || it.qb > q_e[it.e])
          return fail(PUFE_EINVAL, "internal: bad point range in the FP64 work list");
        covered[it.e] += it.qb - it.qa;
        wsplit.push_back(it.e);
        wsplit.push_back(it.qa);
        wsplit.push_back(it.qb);
      }
      for (int64_t e = 0; e < nelem; ++e)
        if (covered[e] != q_e[e])
          return fail(PUFE_EINVAL, "internal: the FP64 work list misses points");
    }
  }
  ctx->n_wsplit = (int64_t)(wsplit.size() / 3);

  // ---- mixed-path work list of the n_e > 128 elements -------------------------
  // The tensor-core kernel runs one persistent CTA per SM over these items; an
  // element's cost is (128-row tiles) x (chunks of 8 padded points).  Elements
  // costing more than the mean per SM are cut into chunk ranges (at least 8
  // chunks each) whose partial tiles meet in the FP64 atomics; the FP32
  // adjoint of these elements takes the same ranges (disjoint points).
  std::vector<int32_t> titems;
  {
    int nsm = 152;
    if (ctx->on_device) {
      int v = 0;
      if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, ctx->device) == cudaSuccess &&
          v > 0)
        nsm = v;
    }
    struct TItem {
      int32_t k, c0, c1;
      int64_t c;
    };
    std::vector<TItem> items;
    int64_t total = 0;
    for (int k = 0; k < n_big; ++k) {
      const int64_t e = order[k];
      total += (int64_t)((n_e[e] + 127) / 128) * ((qpoff[e + 1] - qpoff[e]) / 8);
    }
    const double target = std::max(1.0, (double)total / nsm);
    for (int k = 0; k < n_big; ++k) {
      const int64_t e = order[k];
      const int nmt = (n_e[e] + 127) / 128;
      const int nch = (int)((qpoff[e + 1] - qpoff[e]) / 8);
      int m = (int)std::ceil((double)nmt * nch / target);
      m = std::max(1, std::min(m, nch / 8));
      int prev = 0;
      for (int j = 1; j <= m; ++j) {
        const int b = (j == m) ? nch : (int)((int64_t)j * nch / m);
        items.push_back(TItem{k, prev, b, (int64_t)nmt * (b - prev)});
        prev = b;
      }
    }
    std::stable_sort(items.begin(), items.end(),
                     [](const TItem &x, const TItem &y) { return x.c > y.c; });
    std::vector<int64_t> covered(std::max(1, n_big), 0);
    for (auto &it : items) {
      const int64_t e = order[it.k];
      if (it.c0 < 0 || it.c1 <= it.c0 || (int64_t)it.c1 * 8 > qpoff[e + 1] - qpoff[e])
        return fail(PUFE_EINVAL, "internal: bad chunk range in the mixed work list");
      covered[it.k] += it.c1 - it.c0;
      titems.push_back(it.k);
      titems.push_back(it.c0);
      titems.push_back(it.c1);
    }
    for (int k = 0; k < n_big; ++k)
      if (covered[k] * 8 != qpoff[order[k] + 1] - qpoff[order[k]])
        return fail(PUFE_EINVAL, "internal: the mixed work list misses chunks");
  }
  ctx->n_titems = (int)(titems.size() / 3);

  // Work list of the E-E kernel of S: elements with enrichment columns, cut
  // into ranges of their A (A + 1) / 2 slot pairs so that no range costs
  // (pairs x points) much more than a quarter of the mean per SM (four CTAs
  // share an SM); the ranges' entries are disjoint, so no order is implied.
  std::vector<int32_t> sitems;
  {
    int nsm = 152;
    if (ctx->on_device) {
      int v = 0;
      if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, ctx->device) == cudaSuccess &&
          v > 0)
        nsm = v;
    }
    struct SItem {
      int32_t k, pb, pe;
      int64_t c;
    };
    std::vector<SItem> items;
    int64_t total = 0;
    // elements too large for the projection form's stage whose enrichment
    // slots hold one vertex column each take the Gram form (with more columns
    // per slot the projections, shared by a slot pair's vertex pairs, cost
    // several times fewer operations than the Gram products)
    auto gram = [&](int64_t e) {
      return ctx->see_stage[e] > SEE_STAGE_MAX_F && n_e[e] - 64 <= (int)ealpha[e].size();
    };
    for (int64_t k = 0; k < nelem; ++k) {
      const int64_t e = order[k];
      const int64_t A = (int64_t)ealpha[e].size();
      if (n_e[e] > 64 && !gram(e)) total += A * (A + 1) / 2 * (qoff[e + 1] - qoff[e]);
    }
    const double target = std::max(1.0, (double)total / (4.0 * nsm));
    for (int64_t k = 0; k < nelem; ++k) {
      const int64_t e = order[k];
      if (n_e[e] <= 64 || gram(e)) continue;
      const int A = (int)ealpha[e].size(), np = A * (A + 1) / 2;
      const int64_t Q = qoff[e + 1] - qoff[e];
      const int m = std::max(1, std::min(np, (int)std::ceil((double)np * Q / target)));
      int prev = 0;
      for (int j = 1; j <= m; ++j) {
        const int b = (j == m) ? np : (int)((int64_t)j * np / m);
        items.push_back(SItem{(int32_t)k, prev, b, (int64_t)(b - prev) * Q});
        prev = b;
      }
    }
    std::stable_sort(items.begin(), items.end(),
                     [](const SItem &x, const SItem &y) { return x.c > y.c; });
    for (auto &it : items) {
      sitems.push_back(it.k);
      sitems.push_back(it.pb);
      sitems.push_back(it.pe);
    }
  }
  ctx->n_sitems = (int)(sitems.size() / 3);

  // Gram-form list of the E-E block of S: per element taking that form (see
  // the E-E list above), the
  // lower triangle of (row tile, column tile) pairs of its enrichment columns
  // (tiles of 32 columns when there are at most 32, else 64), each over ranges
  // of GRAM_QCHUNK points whose partial blocks meet in the FP64 atomics
  std::vector<int32_t> gitems32, gitems64;
  for (int64_t k = 0; k < nelem; ++k) {
    const int64_t e = order[k];
    if (n_e[e] <= 64 || ctx->see_stage[e] <= SEE_STAGE_MAX_F ||
        n_e[e] - 64 > (int)ealpha[e].size())
      continue;
    const int nE = n_e[e] - 64;
    const int T = nE <= 32 ? 32 : 64;
    const int nt = (nE + T - 1) / T;
    const int32_t Q = q_e[e];
    std::vector<int32_t> &L = T == 32 ? gitems32 : gitems64;
    for (int rt = 0; rt < nt; ++rt)
      for (int ct = 0; ct <= rt; ++ct)
        for (int32_t qa = 0; qa < Q; qa += GRAM_QCHUNK) {
          L.push_back((int32_t)k);
          L.push_back(rt);
          L.push_back(ct);
          L.push_back(qa);
          L.push_back(std::min<int32_t>(Q, qa + GRAM_QCHUNK));
        }
  }
  ctx->n_gitems32 = (int)(gitems32.size() / 5);
  ctx->n_gitems64 = (int)(gitems64.size() / 5);

  // Work list of the strip kernel (64 < n_e <= 128, after the n_e > 128
  // elements in `order`): an element whose cost (points x enrichment columns)
  // exceeds half the mean per SM (two strip CTAs share an SM) is cut into
  // ranges of its (sub)cells; the ranges' partial blocks meet in the atomics.
  std::vector<int32_t> citems;
  {
    int nsm = 152;
    if (ctx->on_device) {
      int v = 0;
      if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, ctx->device) == cudaSuccess &&
          v > 0)
        nsm = v;
    }
    struct CItem {
      int32_t k, c0, c1;
      int64_t c;
    };
    std::vector<CItem> items;
    auto cell_cost = [&](int64_t e, int32_t j) {
      const int64_t p = part_p[j];
      return p * p * p * (n_e[e] - 64);
    };
    int64_t total = 0;
    for (int64_t k = n_big; k < nelem; ++k) {
      const int64_t e = order[k];
      if (n_e[e] <= 64 || n_e[e] > 128) continue;
      for (int32_t j = partoff[e]; j < partoff[e + 1]; ++j) total += cell_cost(e, j);
    }
    const double target = std::max(1.0, (double)total / (2.0 * nsm));
    for (int64_t k = n_big; k < nelem; ++k) {
      const int64_t e = order[k];
      if (n_e[e] <= 64 || n_e[e] > 128) continue;
      const int32_t nc = partoff[e + 1] - partoff[e];
      int32_t c0 = 0;
      int64_t acc = 0;
      for (int32_t c = 0; c < nc; ++c) {
        const int64_t cc = cell_cost(e, partoff[e] + c);
        if (c > c0 && acc + cc > target) {
          items.push_back(CItem{(int32_t)k, c0, c, acc});
          c0 = c;
          acc = 0;
        }
        acc += cc;
      }
      items.push_back(CItem{(int32_t)k, c0, nc, acc});
    }
    std::stable_sort(items.begin(), items.end(),
                     [](const CItem &x, const CItem &y) { return x.c > y.c; });
    for (auto &it : items) {
      citems.push_back(it.k);
      citems.push_back(it.c0);
      citems.push_back(it.c1);
    }
  }
  ctx->n_citems = (int)(citems.size() / 3);

  // Work list of the FP32 per-point kernels (density; adjoint of the strip in
  // its per-point form): every element, cut into ranges of multiples of 256
  // points so that no range costs (points x basis functions) much more than a
  // quarter of the mean per SM.  Each point is written by one range only.
  std::vector<int32_t> pitems;
  {
    int nsm = 152;
    if (ctx->on_device) {
      int v = 0;
      if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, ctx->device) == cudaSuccess &&
          v > 0)
        nsm = v;
    }
    struct PItem {
      int32_t k, qa, qb;
      int64_t c;
    };
    std::vector<PItem> items;
    int64_t total = 0;
    for (int64_t e = 0; e < nelem; ++e) total += (int64_t)q_e[e] * n_e[e];
    const double target = std::max(1.0, (double)total / (4.0 * nsm));
    for (int64_t k = 0; k < nelem; ++k) {
      const int64_t e = order[k];
      const int32_t Q = q_e[e];
      int m = (int)std::min<double>(std::ceil((double)Q * n_e[e] / target), 1e6);
      m = std::max(1, std::min(m, Q / 256));
      int32_t prev = 0;
      for (int j = 1; j <= m; ++j) {
        const int32_t b = (j == m) ? Q : (int32_t)(((int64_t)j * Q / m) & ~(int64_t)255);
        if (b <= prev) continue;
        items.push_back(PItem{(int32_t)k, prev, b, (int64_t)(b - prev) * n_e[e]});
        prev = b;
      }
    }
    std::stable_sort(items.begin(), items.end(),
                     [](const PItem &x, const PItem &y) { return x.c > y.c; });
    std::vector<int64_t> covered(nelem, 0);
    for (auto &it : items) {
      const int64_t e = order[it.k];
      if (it.qa < 0 || it.qb <= it.qa || it.qb > q_e[e])
        return fail(PUFE_EINVAL, "internal: bad point range in the FP32 per-point work list");
      covered[e] += it.qb - it.qa;
      pitems.push_back(it.k);
      pitems.push_back(it.qa);
      pitems.push_back(it.qb);
    }
    for (int64_t e = 0; e < nelem; ++e)
      if (covered[e] != q_e[e])
        return fail(PUFE_EINVAL, "internal: the FP32 per-point work list misses points");
  }
  ctx->n_pitems = (int)(pitems.size() / 3);

  // CTAs of the FP32 tabulation: TAB_CHUNK table items of one element each
  std::vector<int32_t> tblk(nelem + 1, 0);
  for (int64_t e = 0; e < nelem; ++e) {
    const int64_t items = toff32[e + 1] - toff32[e];
    if (items > INT32_MAX) return fail(PUFE_EINVAL, "element table beyond 32-bit item indices");
    tblk[e + 1] = tblk[e] + (int32_t)((items + TAB_CHUNK - 1) / TAB_CHUNK);
  }
  ctx->n_tblk = tblk[nelem];

  pufe_status st;
  auto &D = ctx->d;
  if (ctx->on_device) {
  if ((st = upload(&D.qoff, qoff)) != PUFE_OK) return st;
  if ((st = upload(&D.x, X)) != PUFE_OK) return st;
  if ((st = upload(&D.w, Wt)) != PUFE_OK) return st;
  if ((st = upload(&D.xi, XI)) != PUFE_OK) return st;
  if ((st = upload(&D.doff, doff)) != PUFE_OK) return st;
  if ((st = upload(&D.dofs, dofs)) != PUFE_OK) return st;
  if ((st = upload(&D.ecol, ecol)) != PUFE_OK) return st;
  if ((st = upload(&D.eshift, eshift)) != PUFE_OK) return st;
  if ((st = upload(&D.aoff, aoff)) != PUFE_OK) return st;
  if ((st = upload(&D.alist, alist)) != PUFE_OK) return st;
  if ((st = upload(&D.toff, toff)) != PUFE_OK) return st;
  if ((st = upload(&D.orb, S.orb)) != PUFE_OK) return st;
  {
    std::vector<OrbitalF> of(S.orb.size());
    for (size_t k = 0; k < S.orb.size(); ++k) {
      const Orbital &o = S.orb[k];
      of[k] = OrbitalF{(float)o.zeta, (float)o.norm, (float)o.rc, (float)(1.0 / o.rc), o.n, o.l, o.m, 0};
    }
    if ((st = upload(&D.orbf, of)) != PUFE_OK) return st;
  }
  if ((st = upload(&D.rowptr, rowptr)) != PUFE_OK) return st;
  if ((st = upload(&D.col, colv)) != PUFE_OK) return st;
  if ((st = upload(&D.soff, soff)) != PUFE_OK) return st;
  if ((st = upload(&D.smap, smap)) != PUFE_OK) return st;
  if ((st = upload(&D.order, order)) != PUFE_OK) return st;
  if (!wsplit.empty() && (st = upload(&D.wsplit, wsplit)) != PUFE_OK) return st;
  if (!titems.empty() && (st = upload(&D.titems, titems)) != PUFE_OK) return st;
  if (!sitems.empty() && (st = upload(&D.sitems, sitems)) != PUFE_OK) return st;
  if (!gitems32.empty() && (st = upload(&D.gitems32, gitems32)) != PUFE_OK) return st;
  if (!gitems64.empty() && (st = upload(&D.gitems64, gitems64)) != PUFE_OK) return st;
  if (!citems.empty() && (st = upload(&D.citems, citems)) != PUFE_OK) return st;
  if (!pitems.empty() && (st = upload(&D.pitems, pitems)) != PUFE_OK) return st;
  if ((st = upload(&D.tblk, tblk)) != PUFE_OK) return st;
  if ((st = upload(&D.eeform, ctx->eeform_host)) != PUFE_OK) return st;
  if (fe_exact) {
    if ((st = upload(&D.Tfe, TF)) != PUFE_OK) return st;
    if ((st = upload(&D.Sfe, SF)) != PUFE_OK) return st;
    if ((st = upload(&D.S0, S0)) != PUFE_OK) return st;
  }
  PUFE_CUDA_TRY(cudaMalloc((void **)&D.psi, std::max<int64_t>(1, ctx->psi_len) * sizeof(double)));
  if ((st = upload(&D.qpoff, qpoff)) != PUFE_OK) return st;
  if ((st = upload(&D.qdat, qdat)) != PUFE_OK) return st;
  if ((st = upload(&D.ptab, ptab)) != PUFE_OK) return st;
  if ((st = upload(&D.partoff, partoff)) != PUFE_OK) return st;
  if ((st = upload(&D.part_p, part_p)) != PUFE_OK) return st;
  if ((st = upload(&D.part_q, part_q)) != PUFE_OK) return st;
  PUFE_CUDA_TRY(cudaMalloc((void **)&D.vpad, std::max<int64_t>(1, qpoff[nelem]) * sizeof(float)));
  if ((st = upload(&D.toff32, toff32)) != PUFE_OK) return st;
  if ((st = upload(&D.eorig, eorig)) != PUFE_OK) return st;
  PUFE_CUDA_TRY(cudaMalloc((void **)&D.psi32, std::max<int64_t>(1, ctx->psi32_len) * sizeof(float)));
  PUFE_CUDA_TRY(cudaMalloc((void **)&D.err, sizeof(unsigned)));
  PUFE_CUDA_TRY(cudaMemset(D.err, 0, sizeof(unsigned)));
  PUFE_CUDA_TRY(cudaStreamCreateWithFlags(&D.side, cudaStreamNonBlocking));
  PUFE_CUDA_TRY(cudaEventCreateWithFlags(&D.ev_fork, cudaEventDisableTiming));
  PUFE_CUDA_TRY(cudaEventCreateWithFlags(&D.ev_join, cudaEventDisableTiming));
  }

  ctx->qoff = std::move(qoff);
  ctx->rowptr = std::move(rowptr);
  ctx->col = std::move(colv);
  ctx->doff = std::move(doff);
  ctx->dofs = std::move(dofs);
  ctx->n_e = std::move(n_e);
  ctx->q_e = std::move(q_e);
  ctx->order = std::move(order);
  ctx->x = std::move(X);
  ctx->w = std::move(Wt);
  return PUFE_OK;
}

static void free_device(pufe_ctx *ctx) {
  scf_free(ctx);
  auto &D = ctx->d;
  void *ptrs[] = {D.qoff, D.x, D.w, D.xi, D.doff, D.dofs, D.ecol, D.eshift, D.aoff, D.alist,
                  D.toff, D.psi, D.psi32, D.qpoff, D.qdat, D.ptab, D.vpad, D.toff32, D.eorig,
                  D.Tfe, D.Sfe, D.S0, D.partoff, D.part_p, D.part_q,
                  D.orb, D.orbf, D.rowptr, D.col, D.soff, D.smap, D.order, D.wsplit,
                  D.titems, D.sitems, D.gitems32, D.gitems64, D.citems, D.pitems, D.tblk, D.eeform, D.err};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  if (D.ev_fork) cudaEventDestroy(D.ev_fork);
  if (D.ev_join) cudaEventDestroy(D.ev_join);
  if (D.side) cudaStreamDestroy(D.side);
  if (D.proj) cudaFree(D.proj);
  D = DeviceArrays();
}

}  // namespace pufe

using namespace pufe;

extern "C" {

pufe_status pufe_build_mesh(const pufe_cell *cell, const pufe_species *species, int nspecies,
                            const pufe_quad *quad, pufe_ctx **out) {
  if (!out) return fail(PUFE_EINVAL, "out must not be NULL");
  *out = nullptr;
  pufe_ctx *ctx = nullptr;
  try {
    ctx = new pufe_ctx();
    pufe_status st = build(cell, species, nspecies, quad, ctx);
    if (st != PUFE_OK) {
      free_device(ctx);
      delete ctx;
      return st;
    }
  } catch (const std::bad_alloc &) {
    if (ctx) {
      free_device(ctx);
      delete ctx;
    }
    return fail(PUFE_ENOMEM, "host allocation failed in pufe_build_mesh");
  } catch (const std::exception &ex) {
    if (ctx) {
      free_device(ctx);
      delete ctx;
    }
    return fail(PUFE_EINVAL, std::string("pufe_build_mesh: ") + ex.what());
  }
  *out = ctx;
  return PUFE_OK;
}

pufe_status pufe_get_sizes(const pufe_ctx *ctx, int64_t *n_dof, int64_t *nnz, int64_t *n_q,
                           int64_t *n_elem, int64_t *max_basis) {
  if (!ctx) return fail(PUFE_EINVAL, "ctx is NULL");
  if (n_dof) *n_dof = ctx->n_dof;
  if (nnz) *nnz = ctx->nnz;
  if (n_q) *n_q = ctx->nq;
  if (n_elem) *n_elem = ctx->nelem;
  if (max_basis) *max_basis = ctx->max_basis;
  return PUFE_OK;
}

pufe_status pufe_get_quadrature(const pufe_ctx *ctx, double *x, double *w,
                                int64_t *elem_offsets) {
  if (!ctx) return fail(PUFE_EINVAL, "ctx is NULL");
  if (x) std::memcpy(x, ctx->x.data(), ctx->x.size() * sizeof(double));
  if (w) std::memcpy(w, ctx->w.data(), ctx->w.size() * sizeof(double));
  if (elem_offsets) std::memcpy(elem_offsets, ctx->qoff.data(), ctx->qoff.size() * sizeof(int64_t));
  return PUFE_OK;
}

pufe_status pufe_get_pattern(const pufe_ctx *ctx, int64_t *rowptr, int32_t *col) {
  if (!ctx) return fail(PUFE_EINVAL, "ctx is NULL");
  if (rowptr) std::memcpy(rowptr, ctx->rowptr.data(), ctx->rowptr.size() * sizeof(int64_t));
  if (col) std::memcpy(col, ctx->col.data(), ctx->col.size() * sizeof(int32_t));
  return PUFE_OK;
}

pufe_status pufe_get_element_basis(const pufe_ctx *ctx, int32_t *n_e, int32_t *dofs) {
  if (!ctx) return fail(PUFE_EINVAL, "ctx is NULL");
  if (n_e) std::memcpy(n_e, ctx->n_e.data(), ctx->n_e.size() * sizeof(int32_t));
  if (dofs) std::memcpy(dofs, ctx->dofs.data(), ctx->dofs.size() * sizeof(int32_t));
  return PUFE_OK;
}

pufe_status pufe_get_element_slots(const pufe_ctx *ctx, int32_t *n_slot) {
  if (!ctx || !n_slot) return fail(PUFE_EINVAL, "ctx and n_slot must not be NULL");
  std::memcpy(n_slot, ctx->n_slot.data(), ctx->n_slot.size() * sizeof(int32_t));
  return PUFE_OK;
}

void pufe_destroy(pufe_ctx *ctx) {
  if (!ctx) return;
  if (!ctx->on_device) {
    delete ctx;
    return;
  }
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(ctx->device);
  for (auto &ev : ctx->pev)
    if (ev) cudaEventDestroy(ev);
  free_device(ctx);
  cudaSetDevice(cur);
  delete ctx;
}

const char *pufe_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
