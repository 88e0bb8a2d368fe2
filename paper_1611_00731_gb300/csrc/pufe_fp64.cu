// FP64 CUDA-core kernels of the PUFE hot path:
//   K0  enrichment tabulation (Sec. 5.1, eqs. Psitilde/Psi)
//   K1+K2+K3  element basis tile, contraction and scatter (Sec. 4, eq. disceig3d)
//   K4  density at quadrature points (Sec. 3, eq. rhoe)
//   K5  adjoint of V -> H (derivative of sum Hbar_ij H_ij with respect to V_q)
//
// The element basis (the FE columns -- 64 tricubic or 32 cubic serendipity
// functions -- then phi_v^PU Psi_alpha columns) is rebuilt on chip from the reference coordinates of each quadrature point
// and the tabulated Psi / grad Psi; it is never stored in HBM.
#include <math.h>

#include "pufe_internal.h"

namespace pufe {

namespace {

constexpr int QC = 8;         // quadrature points per chunk
constexpr int ASM_NT = 256;   // threads of the assembly kernel
constexpr int DEN_NT = 128;   // threads of the density kernel
constexpr int ADJ_NT = 256;   // threads of the adjoint kernel

__device__ __forceinline__ void set_err(unsigned *err, unsigned bit) { atomicOr(err, bit); }

// ---------------------------------------------------------------------------
// K0: Psi and grad Psi for every (enrichment slot, quadrature point) of an element.
// Layout per element: psi[4*toff[e] + (slot*4 + comp)*Q + q].
// ---------------------------------------------------------------------------
// (general cells: `gen` with the lattice `lat`, Sec. 6.2)
__global__ void k_tabulate(const int64_t *__restrict__ qoff, const double *__restrict__ x,
                           const int32_t *__restrict__ aoff, const int32_t *__restrict__ alist,
                           const int64_t *__restrict__ toff, const Orbital *__restrict__ orb,
                           double a0, double a1, double a2, int i0, int i1, int i2,
                           double *__restrict__ psi, int gen, LatticeDev lat) {
  const int64_t e = blockIdx.x;
  const int64_t q0 = qoff[e];
  const int Q = (int)(qoff[e + 1] - q0);
  const int A = aoff[e + 1] - aoff[e];
  const double av[3] = {a0, a1, a2};
  const int img[3] = {i0, i1, i2};
  double *out = psi + 4 * toff[e];
  for (int idx = threadIdx.x; idx < Q * A; idx += blockDim.x) {
    const int slot = idx / Q, q = idx - slot * Q;
    const Orbital o = orb[alist[aoff[e] + slot]];
    const double p[3] = {x[3 * (q0 + q)], x[3 * (q0 + q) + 1], x[3 * (q0 + q) + 2]};
    double v, g[3];
    if (gen)
      enrichment_eval_lat(o, p, lat, v, g);
    else
      enrichment_eval(o, p, av, img, v, g);
    double *dst = out + (int64_t)slot * 4 * Q + q;
    dst[0] = v;
    dst[Q] = g[0];
    dst[2 * Q] = g[1];
    dst[3 * Q] = g[2];
  }
}

// Basis values and physical gradients of column c at reference point xi.
// FE column c: node (c&3, (c>>2)&3, c>>4) from the 1D tables L, dL.
// Enrichment column: PU vertex lv times Psi (value/gradient g4).
struct Tab1D {
  double L[3][4], dL[3][4];
};

__device__ __forceinline__ void fe_column(const Tab1D &t, int c, const double s[3], double &b,
                                          double &gx, double &gy, double &gz) {
  const int ia = c & 3, ib = (c >> 2) & 3, ic = c >> 4;
  const double lx = t.L[0][ia], ly = t.L[1][ib], lz = t.L[2][ic];
  b = lx * ly * lz;
  gx = t.dL[0][ia] * ly * lz * s[0];
  gy = lx * t.dL[1][ib] * lz * s[1];
  gz = lx * ly * t.dL[2][ic] * s[2];
}

__device__ __forceinline__ void pu_column(const double xi[3], int lv, const double s[3],
                                          const double ps[4], double &b, double &gx, double &gy,
                                          double &gz) {
  double h[3], dh[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int bit = (lv >> d) & 1;
    h[d] = bit ? 0.5 * (1.0 + xi[d]) : 0.5 * (1.0 - xi[d]);
    dh[d] = (bit ? 0.5 : -0.5) * s[d];
  }
  const double phi = h[0] * h[1] * h[2];
  b = phi * ps[0];
  gx = dh[0] * h[1] * h[2] * ps[0] + phi * ps[1];
  gy = h[0] * dh[1] * h[2] * ps[0] + phi * ps[2];
  gz = h[0] * h[1] * dh[2] * ps[0] + phi * ps[3];
}

// ---------------------------------------------------------------------------
// K1+K2+K3 (FP64): one CTA per work item -- an element, or with the setup's
// point-range list (`wsplit`) the points [qa, qb) of one.  Per chunk of QC
// points the CTA builds y_d = sqrt(w/2) G_d, z = sqrt(w) B and zv = V z in
// shared memory; each thread owns 4x4 blocks of the lower triangle and
// accumulates
//   H += sum_d y_d y_d^T + zv z^T,   S += z z^T,
// over the item's points, then adds its entries into the CSR values through
// the scatter map (the ranges of one element meet in these atomics).
// ---------------------------------------------------------------------------
// BLOCH: the scatter carries the phase exp(i k.(R_j - R_i)) of the column
// pair (lattice shifts from `eshift`, phases of the 8 shift codes in `ph`)
// into separate real and imaginary outputs (Sec. 4, eq. bloch).  GEN: a
// general cell, physical gradients J^-T grad_xi with jit = J^-T (row-major).
struct Mat3 {
  double m[9];
};

template <bool BLOCH, bool GEN>
__global__ void __launch_bounds__(ASM_NT) k_assemble_fp64(
    const int32_t *__restrict__ order, const int64_t *__restrict__ qoff,
    const double *__restrict__ w, const double *__restrict__ xi_all,
    const int64_t *__restrict__ doff, const int32_t *__restrict__ ecol,
    const int64_t *__restrict__ toff, const double *__restrict__ psi,
    const int64_t *__restrict__ soff, const int32_t *__restrict__ smap,
    const double *__restrict__ V, double sx, double sy, double sz, int npad_max, int want,
    double *__restrict__ H, double *__restrict__ S, unsigned *err,
    const uint8_t *__restrict__ eshift, PhaseTab ph, double *__restrict__ Hi,
    double *__restrict__ Si, const int32_t *__restrict__ wsplit, Mat3 jit, int nfe) {
  extern __shared__ __align__(16) double smem[];
  // work item: a whole element, or the point range [qa, qb) of one
  const int e = wsplit ? wsplit[3 * blockIdx.x] : order[blockIdx.x];
  const int64_t q0 = qoff[e];
  const int Q = (int)(qoff[e + 1] - q0);
  const int qa = wsplit ? max(wsplit[3 * blockIdx.x + 1], 0) : 0;
  const int qb = wsplit ? min(wsplit[3 * blockIdx.x + 2], Q) : Q;
  const int n = (int)(doff[e + 1] - doff[e]);
  const int npad = (n + 3) & ~3;
  if (npad > npad_max) {
    if (threadIdx.x == 0) set_err(err, DEVERR_SHAPE);
    return;
  }
  const int32_t *ec = ecol + (doff[e] - (int64_t)nfe * e);
  const double *pe = psi + 4 * toff[e];
  // shared layout: 5 arrays [QC][npad] then 1D tables
  double *Y0 = smem, *Y1 = Y0 + QC * npad, *Y2 = Y1 + QC * npad, *Z = Y2 + QC * npad,
         *ZV = Z + QC * npad;
  Tab1D *tab = reinterpret_cast<Tab1D *>(ZV + QC * npad);
  const double s[3] = {sx, sy, sz};

  const int nb = npad / 4;
  const int nblk = nb * (nb + 1) / 2;
  for (int base = 0; base < nblk; base += ASM_NT) {
    const int t = base + threadIdx.x;
    const bool active = t < nblk;
    int I = 0, J = 0;
    if (active) {
      I = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
      while ((I + 1) * (I + 2) / 2 <= t) ++I;
      while (I * (I + 1) / 2 > t) --I;
      J = t - I * (I + 1) / 2;
    }
    const int i0 = 4 * I, j0 = 4 * J;
    double h[4][4], sv[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) h[a][b] = sv[a][b] = 0.0;

    for (int qc = qa; qc < qb; qc += QC) {
      __syncthreads();
      // 1D Lagrange tables of the chunk's points
      for (int k = threadIdx.x; k < QC * 3; k += ASM_NT) {
        const int qq = k / 3, d = k - 3 * qq;
        const int q = qc + qq;
        const double xv = (q < qb) ? xi_all[3 * (q0 + q) + d] : 0.0;
        double L[4], dL[4];
        lagrange3(xv, L, dL);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          tab[qq].L[d][c] = L[c];
          tab[qq].dL[d][c] = dL[c];
        }
      }
      __syncthreads();
      for (int k = threadIdx.x; k < QC * npad; k += ASM_NT) {
        const int qq = k / npad, c = k - qq * npad;
        const int q = qc + qq;
        double b = 0, gx = 0, gy = 0, gz = 0, sw = 0, vv = 0;
        if (q < qb && c < n) {
          // GEN: reference gradients (unit scales) mapped by J^-T
          const double one[3] = {1.0, 1.0, 1.0};
          auto tomap = [&](double &x, double &y, double &z) {
            const double rx = x, ry = y, rz = z;
            x = jit.m[0] * rx + jit.m[1] * ry + jit.m[2] * rz;
            y = jit.m[3] * rx + jit.m[4] * ry + jit.m[5] * rz;
            z = jit.m[6] * rx + jit.m[7] * ry + jit.m[8] * rz;
          };
          if (c < nfe) {   // FE column: tricubic (64) or serendipity (32)
            if (nfe == 64) {
              fe_column(tab[qq], c, GEN ? one : s, b, gx, gy, gz);
            } else {
              const double xq[3] = {xi_all[3 * (q0 + q)], xi_all[3 * (q0 + q) + 1],
                                    xi_all[3 * (q0 + q) + 2]};
              const double *sc = GEN ? one : s;
              double g3[3];
              serendipity32(c, xq, b, g3);
              gx = g3[0] * sc[0];
              gy = g3[1] * sc[1];
              gz = g3[2] * sc[2];
            }
            if (GEN) tomap(gx, gy, gz);
          } else {
            const int code = ec[c - nfe];
            const int slot = code >> 3, lv = code & 7;
            const double *pp = pe + (int64_t)slot * 4 * Q + q;
            const double ps[4] = {pp[0], pp[Q], pp[2 * Q], pp[3 * Q]};
            const double xq[3] = {xi_all[3 * (q0 + q)], xi_all[3 * (q0 + q) + 1],
                                  xi_all[3 * (q0 + q) + 2]};
            if (GEN) {   // phi_v and its mapped gradient, then the product rule
              const double unit[4] = {1.0, 0.0, 0.0, 0.0};
              double phi;
              pu_column(xq, lv, one, unit, phi, gx, gy, gz);
              tomap(gx, gy, gz);
              b = phi * ps[0];
              gx = gx * ps[0] + phi * ps[1];
              gy = gy * ps[0] + phi * ps[2];
              gz = gz * ps[0] + phi * ps[3];
            } else {
              pu_column(xq, lv, s, ps, b, gx, gy, gz);
            }
          }
          sw = w[q0 + q];
          vv = V ? V[q0 + q] : 0.0;
          if (!isfinite(vv)) atomicOr(err, DEVERR_NONFINITE);
        }
        const double r2 = sqrt(0.5 * sw), r1 = sqrt(sw);
        Y0[k] = r2 * gx;
        Y1[k] = r2 * gy;
        Y2[k] = r2 * gz;
        Z[k] = r1 * b;
        ZV[k] = vv * r1 * b;
      }
      __syncthreads();
      if (active) {
        const int qn = min(QC, qb - qc);
        for (int qq = 0; qq < qn; ++qq) {
          const int ro = qq * npad;
          double ai[5][4], bj[4][4];
#pragma unroll
          for (int a = 0; a < 4; ++a) {
            ai[0][a] = Y0[ro + i0 + a];
            ai[1][a] = Y1[ro + i0 + a];
            ai[2][a] = Y2[ro + i0 + a];
            ai[3][a] = ZV[ro + i0 + a];
            ai[4][a] = Z[ro + i0 + a];
            bj[0][a] = Y0[ro + j0 + a];
            bj[1][a] = Y1[ro + j0 + a];
            bj[2][a] = Y2[ro + j0 + a];
            bj[3][a] = Z[ro + j0 + a];
          }
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) {
              double acc = h[a][b];
              acc = fma(ai[0][a], bj[0][b], acc);
              acc = fma(ai[1][a], bj[1][b], acc);
              acc = fma(ai[2][a], bj[2][b], acc);
              acc = fma(ai[3][a], bj[3][b], acc);
              h[a][b] = acc;
              sv[a][b] = fma(ai[4][a], bj[3][b], sv[a][b]);
            }
        }
      }
    }
    // scatter the owned lower-triangle entries (both (i,j) and (j,i))
    if (active) {
      const int32_t *m = smap + soff[e];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const int i = i0 + a, j = j0 + b;
          if (i >= n || j >= n || j > i) continue;
          const int32_t sij = m[(int64_t)i * n + j];
          const int32_t sji = m[(int64_t)j * n + i];
          if (BLOCH) {
            // (i, j) gets conj(ph_i) ph_j, (j, i) its conjugate
            const int ci = eshift[doff[e] + i], cj = eshift[doff[e] + j];
            double pr = 1.0, pim = 0.0;
            if (ci != cj) {
              pr = ph.re[ci] * ph.re[cj] + ph.im[ci] * ph.im[cj];
              pim = ph.re[ci] * ph.im[cj] - ph.im[ci] * ph.re[cj];
            }
            if (want & PUFE_WANT_H) {
              atomicAdd(H + sij, h[a][b] * pr);
              atomicAdd(Hi + sij, h[a][b] * pim);
              if (i != j) {
                atomicAdd(H + sji, h[a][b] * pr);
                atomicAdd(Hi + sji, -h[a][b] * pim);
              }
            }
            if (want & PUFE_WANT_S) {
              atomicAdd(S + sij, sv[a][b] * pr);
              atomicAdd(Si + sij, sv[a][b] * pim);
              if (i != j) {
                atomicAdd(S + sji, sv[a][b] * pr);
                atomicAdd(Si + sji, -sv[a][b] * pim);
              }
            }
            continue;
          }
          if (want & PUFE_WANT_H) {
            atomicAdd(H + sij, h[a][b]);
            if (i != j) atomicAdd(H + sji, h[a][b]);
          }
          if (want & PUFE_WANT_S) {
            atomicAdd(S + sij, sv[a][b]);
            if (i != j) atomicAdd(S + sji, sv[a][b]);
          }
        }
    }
  }
}

// ---------------------------------------------------------------------------
// K4 (FP64): one CTA per element, one thread per quadrature point.  The
// element's coefficient block C_e (n x nocc, gathered through the element DOF
// list) sits in shared memory; each thread evaluates its basis row on the fly.
// ---------------------------------------------------------------------------
template <int KC, bool SER>
__device__ __forceinline__ double density_point(const double xi[3], int q, int Q, int nenr,
                                                const int32_t *ec, const double *pe,
                                                const double *Cs, const double *fs, int nocc,
                                                int k0) {
  double acc[KC];
#pragma unroll
  for (int k = 0; k < KC; ++k) acc[k] = 0.0;
  constexpr int NF = SER ? 32 : 64;
  if (SER) {   // the 32 serendipity columns
    for (int c = 0; c < 32; ++c) {
      double b, g3[3];
      serendipity32(c, xi, b, g3);
      const double *cr = Cs + c * nocc + k0;
#pragma unroll
      for (int k = 0; k < KC; ++k) acc[k] = fma(b, cr[k], acc[k]);
    }
  } else {
    double L[3][4], dL[3][4];
#pragma unroll
    for (int d = 0; d < 3; ++d) lagrange3(xi[d], L[d], dL[d]);
#pragma unroll
    for (int c3 = 0; c3 < 4; ++c3)
#pragma unroll
      for (int c2 = 0; c2 < 4; ++c2) {
        const double lyz = L[1][c2] * L[2][c3];
#pragma unroll
        for (int c1 = 0; c1 < 4; ++c1) {
          const double b = L[0][c1] * lyz;
          const double *cr = Cs + (c1 + 4 * c2 + 16 * c3) * nocc + k0;
#pragma unroll
          for (int k = 0; k < KC; ++k) acc[k] = fma(b, cr[k], acc[k]);
        }
      }
  }
  for (int j = 0; j < nenr; ++j) {
    const int code = ec[j];
    const int slot = code >> 3, lv = code & 7;
    double phi = 1.0;
#pragma unroll
    for (int d = 0; d < 3; ++d) phi *= ((lv >> d) & 1) ? 0.5 * (1.0 + xi[d]) : 0.5 * (1.0 - xi[d]);
    const double b = phi * pe[(int64_t)slot * 4 * Q + q];
    const double *cr = Cs + (NF + j) * nocc + k0;
#pragma unroll
    for (int k = 0; k < KC; ++k) acc[k] = fma(b, cr[k], acc[k]);
  }
  double r = 0.0;
#pragma unroll
  for (int k = 0; k < KC; ++k) r = fma(fs[k0 + k] * acc[k], acc[k], r);
  return r;
}

// BLOCH: complex coefficients C + i Ci; each element block is gathered with
// the column phases applied, and n = sum_k f_k (Re psi_k^2 + Im psi_k^2).
template <bool BLOCH, bool SER>
__global__ void __launch_bounds__(DEN_NT) k_density_fp64(
    const int32_t *__restrict__ order, const int64_t *__restrict__ qoff,
    const double *__restrict__ xi_all, const int64_t *__restrict__ doff,
    const int32_t *__restrict__ dofs, const int32_t *__restrict__ ecol,
    const int64_t *__restrict__ toff, const double *__restrict__ psi,
    const double *__restrict__ C, int64_t ldc, const double *__restrict__ f, int nocc,
    int noccp, double *__restrict__ rho, const uint8_t *__restrict__ eshift, PhaseTab ph,
    const double *__restrict__ Ci) {
  extern __shared__ __align__(16) double smem[];
  const int e = order[blockIdx.x];
  const int64_t q0 = qoff[e];
  const int Q = (int)(qoff[e + 1] - q0);
  const int n = (int)(doff[e + 1] - doff[e]);
  constexpr int NF = SER ? 32 : 64;   // FE columns
  const int nenr = n - NF;
  const int32_t *ec = ecol + (doff[e] - (int64_t)NF * e);
  const int32_t *dl = dofs + doff[e];
  const double *pe = psi + 4 * toff[e];
  double *Cs = smem;             // n x noccp
  double *fs = Cs + n * noccp;   // noccp
  double *Cz = fs + noccp;       // n x noccp, imaginary parts (BLOCH)
  for (int k = threadIdx.x; k < n * noccp; k += DEN_NT) {
    const int j = k / noccp, kk = k - j * noccp;
    if (BLOCH) {
      double cr = 0.0, ci = 0.0;
      if (kk < nocc) {
        const double ar = C[(int64_t)dl[j] * ldc + kk], ai = Ci[(int64_t)dl[j] * ldc + kk];
        const int c = eshift[doff[e] + j];
        cr = ph.re[c] * ar - ph.im[c] * ai;
        ci = ph.re[c] * ai + ph.im[c] * ar;
      }
      Cs[k] = cr;
      Cz[k] = ci;
    } else {
      Cs[k] = (kk < nocc) ? C[(int64_t)dl[j] * ldc + kk] : 0.0;
    }
  }
  for (int k = threadIdx.x; k < noccp; k += DEN_NT) fs[k] = (k < nocc) ? f[k] : 0.0;
  __syncthreads();
  for (int q = threadIdx.x; q < Q; q += DEN_NT) {
    const double xq[3] = {xi_all[3 * (q0 + q)], xi_all[3 * (q0 + q) + 1], xi_all[3 * (q0 + q) + 2]};
    double r = 0.0;
    for (int k0 = 0; k0 < noccp; k0 += 8) {
      r += density_point<8, SER>(xq, q, Q, nenr, ec, pe, Cs, fs, noccp, k0);
      if (BLOCH) r += density_point<8, SER>(xq, q, Q, nenr, ec, pe, Cz, fs, noccp, k0);
    }
    rho[q0 + q] = r;
  }
}

// ---------------------------------------------------------------------------
// K5 (FP64): Vbar_q = w_q b_q^T Hbar_e b_q.  One CTA per work item (an
// element, or the point range [qa, qb) of one, as in the assembly): the
// element block Hbar_e is gathered into shared memory (or read through the
// scatter map when it does not fit); per chunk of QC points the basis rows are
// built in shared memory and each thread reduces one (q, i) pair over j.
// ---------------------------------------------------------------------------
// BLOCH: complex cotangent Hbar + i Hbi; the element block used is
// Re(conj(Hbar) exp(i k.(R_j - R_i))) = Hbar pr + Hbi pi.
template <bool BLOCH>
__global__ void __launch_bounds__(ADJ_NT) k_adjoint_fp64(
    const int32_t *__restrict__ order, const int64_t *__restrict__ qoff,
    const double *__restrict__ w, const double *__restrict__ xi_all,
    const int64_t *__restrict__ doff, const int32_t *__restrict__ ecol,
    const int64_t *__restrict__ toff, const double *__restrict__ psi,
    const int64_t *__restrict__ soff, const int32_t *__restrict__ smap,
    const double *__restrict__ Hbar, int hs_in_smem, double *__restrict__ Vbar,
    const uint8_t *__restrict__ eshift, PhaseTab ph, const double *__restrict__ Hbi,
    const int32_t *__restrict__ wsplit, int nfe) {
  extern __shared__ __align__(16) double smem[];
  // work item: a whole element, or the point range [qa, qb) of one
  const int e = wsplit ? wsplit[3 * blockIdx.x] : order[blockIdx.x];
  const int64_t q0 = qoff[e];
  const int Q = (int)(qoff[e + 1] - q0);
  const int qa = wsplit ? max(wsplit[3 * blockIdx.x + 1], 0) : 0;
  const int qb = wsplit ? min(wsplit[3 * blockIdx.x + 2], Q) : Q;
  const int n = (int)(doff[e + 1] - doff[e]);
  const int32_t *ec = ecol + (doff[e] - (int64_t)nfe * e);
  const double *pe = psi + 4 * toff[e];
  const int32_t *m = smap + soff[e];
  double *Bc = smem;                 // QC x n
  double *acc = Bc + QC * n;         // QC
  Tab1D *tab = reinterpret_cast<Tab1D *>(acc + QC);
  double *Hs = reinterpret_cast<double *>(tab + QC);  // n x n when it fits
  // element entry (i, j) of the cotangent (phased real part for BLOCH)
  auto hval = [&](int i, int j) -> double {
    const int32_t sl = m[(int64_t)i * n + j];
    if (!BLOCH) return Hbar[sl];
    const int ci = eshift[doff[e] + i], cj = eshift[doff[e] + j];
    double pr = 1.0, pim = 0.0;
    if (ci != cj) {
      pr = ph.re[ci] * ph.re[cj] + ph.im[ci] * ph.im[cj];
      pim = ph.re[ci] * ph.im[cj] - ph.im[ci] * ph.re[cj];
    }
    return Hbar[sl] * pr + Hbi[sl] * pim;
  };
  if (hs_in_smem)
    for (int k = threadIdx.x; k < n * n; k += ADJ_NT) Hs[k] = hval(k / n, k % n);
  const double s[3] = {0, 0, 0};
  for (int qc = qa; qc < qb; qc += QC) {
    __syncthreads();
    for (int k = threadIdx.x; k < QC * 3; k += ADJ_NT) {
      const int qq = k / 3, d = k - 3 * qq;
      const int q = qc + qq;
      const double xv = (q < qb) ? xi_all[3 * (q0 + q) + d] : 0.0;
      double L[4], dL[4];
      lagrange3(xv, L, dL);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        tab[qq].L[d][c] = L[c];
        tab[qq].dL[d][c] = dL[c];
      }
    }
    if (threadIdx.x < QC) acc[threadIdx.x] = 0.0;
    __syncthreads();
    for (int k = threadIdx.x; k < QC * n; k += ADJ_NT) {
      const int qq = k / n, c = k - qq * n;
      const int q = qc + qq;
      double b = 0, gx, gy, gz;
      if (q < qb) {
        if (c < nfe) {   // FE column: tricubic (64) or serendipity (32)
          if (nfe == 64) {
            fe_column(tab[qq], c, s, b, gx, gy, gz);
          } else {
            const double xq[3] = {xi_all[3 * (q0 + q)], xi_all[3 * (q0 + q) + 1],
                                  xi_all[3 * (q0 + q) + 2]};
            double g3[3];
            serendipity32(c, xq, b, g3);
          }
        } else {
          const int code = ec[c - nfe];
          const int slot = code >> 3, lv = code & 7;
          const double *pp = pe + (int64_t)slot * 4 * Q + q;
          const double ps[4] = {pp[0], 0.0, 0.0, 0.0};
          const double xq[3] = {xi_all[3 * (q0 + q)], xi_all[3 * (q0 + q) + 1],
                                xi_all[3 * (q0 + q) + 2]};
          pu_column(xq, lv, s, ps, b, gx, gy, gz);
        }
      }
      Bc[k] = b;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < QC * n; k += ADJ_NT) {
      const int qq = k / n, i = k - qq * n;
      if (qc + qq >= qb) continue;
      const double *brow = Bc + qq * n;
      double t = 0.0;
      if (hs_in_smem) {
        const double *hr = Hs + (int64_t)i * n;
        for (int j = 0; j < n; ++j) t = fma(hr[j], brow[j], t);
      } else {
        for (int j = 0; j < n; ++j) t = fma(hval(i, j), brow[j], t);
      }
      atomicAdd(acc + qq, brow[i] * t);
    }
    __syncthreads();
    if (threadIdx.x < QC && qc + (int)threadIdx.x < qb)
      Vbar[q0 + qc + threadIdx.x] = w[q0 + qc + threadIdx.x] * acc[threadIdx.x];
  }
}

// ---------------------------------------------------------------------------
// Projections of the basis onto separable nonlocal projectors (Sec. 4):
// F[g_i, p] = sum_e sum_q w_q b_i(x_q) v_p(x_q), with the Gaussian projectors
// v_p = N r^l exp(-r^2 / (2 r_p^2)) Y_lm summed over the periodic images
// within r_cut.  One CTA per element; per chunk of QC points the basis rows
// and w v_p go to shared memory; the element's n x P block accumulates in
// shared memory and is added into F at the end.
// BLOCH (Sec. 4, eqs. bloch, strong): the image at lattice vector a_n carries
// exp(i k.a_n) and column i of the element the factor exp(-i k.R_i) of its
// lattice shift R_i, so F is complex (real and imaginary N x P arrays).
// ---------------------------------------------------------------------------
template <bool BLOCH>
__global__ void __launch_bounds__(ASM_NT) k_projections(
    const int64_t *__restrict__ qoff, const double *__restrict__ w,
    const double *__restrict__ xi_all, const double *__restrict__ x,
    const int64_t *__restrict__ doff, const int32_t *__restrict__ dofs,
    const int32_t *__restrict__ ecol, const int64_t *__restrict__ toff,
    const double *__restrict__ psi, const ProjDev *__restrict__ pj, int P, double a0, double a1,
    double a2, double *__restrict__ F, const uint8_t *__restrict__ eshift, PhaseTab ph,
    double k0, double k1, double k2, double *__restrict__ Fi) {
  extern __shared__ __align__(16) double smem[];
  constexpr int NC = BLOCH ? 2 : 1;   // real, imaginary parts
  const int e = blockIdx.x;
  const int64_t q0 = qoff[e];
  const int Q = (int)(qoff[e + 1] - q0);
  const int n = (int)(doff[e + 1] - doff[e]);
  const int32_t *ec = ecol + (doff[e] - 64ll * e);
  const double *pe = psi + 4 * toff[e];
  double *Bc = smem;               // QC x n
  double *Vp = Bc + QC * n;        // [NC] QC x P
  double *acc = Vp + NC * QC * P;  // [NC] n x P
  Tab1D *tab = reinterpret_cast<Tab1D *>(acc + (size_t)NC * n * P);
  const double av[3] = {a0, a1, a2};
  const double s[3] = {0, 0, 0};
  for (int k = threadIdx.x; k < NC * n * P; k += ASM_NT) acc[k] = 0.0;
  for (int qc = 0; qc < Q; qc += QC) {
    __syncthreads();
    for (int k = threadIdx.x; k < QC * 3; k += ASM_NT) {
      const int qq = k / 3, d = k - 3 * qq;
      const int q = qc + qq;
      const double xv = (q < Q) ? xi_all[3 * (q0 + q) + d] : 0.0;
      double L[4], dL[4];
      lagrange3(xv, L, dL);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        tab[qq].L[d][c] = L[c];
        tab[qq].dL[d][c] = dL[c];
      }
    }
    for (int k = threadIdx.x; k < QC * P; k += ASM_NT) {
      const int qq = k / P, p = k - qq * P;
      const int q = qc + qq;
      double v = 0.0, vi = 0.0;
      if (q < Q) {
        const ProjDev pr = pj[p];
        double d[3];
        int lo[3], hi[3];
        for (int c = 0; c < 3; ++c) {
          d[c] = x[3 * (q0 + q) + c] - pr.tau[c];
          lo[c] = (int)ceil((-pr.rcut - d[c]) / av[c]);
          hi[c] = (int)floor((pr.rcut - d[c]) / av[c]);
        }
        const double i2 = 1.0 / (2.0 * pr.rp * pr.rp);
        for (int i = lo[0]; i <= hi[0]; ++i)
          for (int j = lo[1]; j <= hi[1]; ++j)
            for (int l = lo[2]; l <= hi[2]; ++l) {
              const double dx = d[0] + i * av[0], dy = d[1] + j * av[1], dz = d[2] + l * av[2];
              const double r2 = dx * dx + dy * dy + dz * dz;
              if (r2 >= pr.rcut * pr.rcut) continue;
              double g[3];
              const double val = pr.N * exp(-r2 * i2) * solid_harmonic(pr.l, pr.m, dx, dy, dz, g);
              if (BLOCH) {   // exp(i k.a_n): this term is v(x - tau - a_n), a_n = -(i a0, j a1, l a2)
                double sn, cs;
                sincos(-(k0 * (i * av[0]) + k1 * (j * av[1]) + k2 * (l * av[2])), &sn, &cs);
                v += val * cs;
                vi += val * sn;
              } else {
                v += val;
              }
            }
        v *= w[q0 + q];
        vi *= w[q0 + q];
      }
      Vp[k] = v;
      if (BLOCH) Vp[QC * P + k] = vi;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < QC * n; k += ASM_NT) {
      const int qq = k / n, c = k - qq * n;
      const int q = qc + qq;
      double b = 0, gx, gy, gz;
      if (q < Q) {
        if (c < 64) {
          fe_column(tab[qq], c, s, b, gx, gy, gz);
        } else {
          const int code = ec[c - 64];
          const int slot = code >> 3, lv = code & 7;
          const double ps[4] = {pe[(int64_t)slot * 4 * Q + q], 0.0, 0.0, 0.0};
          const double xq[3] = {xi_all[3 * (q0 + q)], xi_all[3 * (q0 + q) + 1],
                                xi_all[3 * (q0 + q) + 2]};
          pu_column(xq, lv, s, ps, b, gx, gy, gz);
        }
      }
      Bc[k] = b;
    }
    __syncthreads();
    const int qn = min(QC, Q - qc);
    for (int k = threadIdx.x; k < n * P; k += ASM_NT) {
      const int i = k / P, p = k - i * P;
      double t = acc[k], ti = BLOCH ? acc[n * P + k] : 0.0;
      for (int qq = 0; qq < qn; ++qq) {
        t = fma(Bc[qq * n + i], Vp[qq * P + p], t);
        if (BLOCH) ti = fma(Bc[qq * n + i], Vp[QC * P + qq * P + p], ti);
      }
      acc[k] = t;
      if (BLOCH) acc[n * P + k] = ti;
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < n * P; k += ASM_NT) {
    const int i = k / P, p = k - i * P;
    const int64_t o = (int64_t)dofs[doff[e] + i] * P + p;
    if (BLOCH) {   // times conj(exp(i k.R_i))
      const int c = eshift[doff[e] + i];
      const double cr = ph.re[c], ci = -ph.im[c], ar = acc[k], ai = acc[n * P + k];
      atomicAdd(F + o, cr * ar - ci * ai);
      atomicAdd(Fi + o, cr * ai + ci * ar);
    } else {
      atomicAdd(F + o, acc[k]);
    }
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
// the lattice of a general cell for the image sums
static LatticeDev lattice_of(const pufe_ctx *ctx) {
  LatticeDev l{};
  if (!ctx->general) return l;
  const double *L = ctx->lat;
  for (int k = 0; k < 9; ++k) l.L[k] = L[k];
  const double det = L[0] * (L[4] * L[8] - L[5] * L[7]) - L[1] * (L[3] * L[8] - L[5] * L[6]) +
                     L[2] * (L[3] * L[7] - L[4] * L[6]);
  const double C[9] = {L[4] * L[8] - L[5] * L[7], L[5] * L[6] - L[3] * L[8],
                       L[3] * L[7] - L[4] * L[6], L[2] * L[7] - L[1] * L[8],
                       L[0] * L[8] - L[2] * L[6], L[1] * L[6] - L[0] * L[7],
                       L[1] * L[5] - L[2] * L[4], L[2] * L[3] - L[0] * L[5],
                       L[0] * L[4] - L[1] * L[3]};
  for (int k = 0; k < 9; ++k) l.Lit[k] = C[k] / det;
  for (int k = 0; k < 3; ++k) l.img[k] = ctx->images[k];
  return l;
}

static Mat3 jit_of(const pufe_ctx *ctx) {
  Mat3 m{};
  for (int k = 0; k < 9; ++k) m.m[k] = ctx->Jit[k];
  return m;
}

pufe_status launch_tabulate(pufe_ctx *ctx, cudaStream_t st) {
  if (ctx->psi_len == 0) return PUFE_OK;
  auto &D = ctx->d;
  k_tabulate<<<(unsigned)ctx->nelem, 128, 0, st>>>(D.qoff, D.x, D.aoff, D.alist, D.toff, D.orb,
                                                   ctx->a[0], ctx->a[1], ctx->a[2],
                                                   ctx->images[0], ctx->images[1], ctx->images[2],
                                                   D.psi, ctx->general ? 1 : 0, lattice_of(ctx));
  PUFE_CUDA_TRY(cudaGetLastError());
  return PUFE_OK;
}

// CTAs of the FP64 assembly and adjoint: one per work item of the point-range
// list when the setup made one, else one per element
static unsigned fp64_items(const pufe_ctx *ctx) {
  return ctx->d.wsplit ? (unsigned)ctx->n_wsplit : (unsigned)ctx->nelem;
}

pufe_status launch_assemble_fp64(pufe_ctx *ctx, const double *V, int what, double *H, double *S,
                                 cudaStream_t st) {
  auto &D = ctx->d;
  const int npad = (ctx->max_basis + 3) & ~3;
  const size_t sm = (size_t)5 * QC * npad * sizeof(double) + QC * sizeof(Tab1D);
  if (sm > 227 * 1024) return fail(PUFE_EINVAL, "element basis too large for the FP64 kernel");
  auto kern = ctx->general ? k_assemble_fp64<false, true> : k_assemble_fp64<false, false>;
  PUFE_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  kern<<<fp64_items(ctx), ASM_NT, sm, st>>>(
      D.order, D.qoff, D.w, D.xi, D.doff, D.ecol, D.toff, D.psi, D.soff, D.smap, V,
      2.0 / ctx->h[0], 2.0 / ctx->h[1], 2.0 / ctx->h[2], npad, what, H, S, D.err, nullptr,
      PhaseTab{}, nullptr, nullptr, D.wsplit, jit_of(ctx), ctx->nfe_e);
  PUFE_CUDA_TRY(cudaGetLastError());
  return PUFE_OK;
}

pufe_status launch_density_fp64(pufe_ctx *ctx, const double *C, int64_t ldc, const double *f,
                                int nocc, double *rho, cudaStream_t st) {
  auto &D = ctx->d;
  const int noccp = (nocc + 7) & ~7;
  const size_t sm = ((size_t)ctx->max_basis * noccp + noccp) * sizeof(double);
  if (sm > 227 * 1024) return fail(PUFE_EINVAL, "n_e * nocc too large for the density kernel");
  auto kern = ctx->ser ? k_density_fp64<false, true> : k_density_fp64<false, false>;
  PUFE_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  kern<<<(unsigned)ctx->nelem, DEN_NT, sm, st>>>(
      D.order, D.qoff, D.xi, D.doff, D.dofs, D.ecol, D.toff, D.psi, C, ldc, f, nocc, noccp, rho,
      nullptr, PhaseTab{}, nullptr);
  PUFE_CUDA_TRY(cudaGetLastError());
  return PUFE_OK;
}

pufe_status launch_adjoint_fp64(pufe_ctx *ctx, const double *Hbar, double *Vbar, cudaStream_t st) {
  auto &D = ctx->d;
  const int n = ctx->max_basis;
  size_t sm = (size_t)QC * n * sizeof(double) + QC * sizeof(double) + QC * sizeof(Tab1D);
  const size_t hs = (size_t)n * n * sizeof(double);
  int in_smem = (sm + hs <= 200 * 1024) ? 1 : 0;
  if (in_smem) sm += hs;
  PUFE_CUDA_TRY(cudaFuncSetAttribute(k_adjoint_fp64<false>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  k_adjoint_fp64<false><<<fp64_items(ctx), ADJ_NT, sm, st>>>(
      D.order, D.qoff, D.w, D.xi, D.doff, D.ecol, D.toff, D.psi, D.soff, D.smap, Hbar, in_smem,
      Vbar, nullptr, PhaseTab{}, nullptr, D.wsplit, ctx->nfe_e);
  PUFE_CUDA_TRY(cudaGetLastError());
  return PUFE_OK;
}

// ---------------------------------------------------------------------------
// Bloch (k != 0) launchers
// ---------------------------------------------------------------------------
PhaseTab phase_table(const pufe_ctx *ctx, const double k[3]) {
  PhaseTab t;
  for (int c = 0; c < 8; ++c) {
    double th = 0.0;
    for (int d = 0; d < 3; ++d)
      if ((c >> d) & 1) {
        if (ctx->general)   // the lattice vector a_d
          th += k[0] * ctx->lat[3 * d] + k[1] * ctx->lat[3 * d + 1] + k[2] * ctx->lat[3 * d + 2];
        else
          th += k[d] * ctx->a[d];
      }
    t.re[c] = cos(th);
    t.im[c] = sin(th);
  }
  return t;
}

pufe_status launch_assemble_fp64_bloch(pufe_ctx *ctx, const PhaseTab &ph, const double *V,
                                       int what, double *H, double *Hi, double *S, double *Si,
                                       cudaStream_t st) {
  auto &D = ctx->d;
  const int npad = (ctx->max_basis + 3) & ~3;
  const size_t sm = (size_t)5 * QC * npad * sizeof(double) + QC * sizeof(Tab1D);
  if (sm > 227 * 1024) return fail(PUFE_EINVAL, "element basis too large for the FP64 kernel");
  auto kern = ctx->general ? k_assemble_fp64<true, true> : k_assemble_fp64<true, false>;
  PUFE_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  kern<<<fp64_items(ctx), ASM_NT, sm, st>>>(
      D.order, D.qoff, D.w, D.xi, D.doff, D.ecol, D.toff, D.psi, D.soff, D.smap, V,
      2.0 / ctx->h[0], 2.0 / ctx->h[1], 2.0 / ctx->h[2], npad, what, H, S, D.err, D.eshift, ph,
      Hi, Si, D.wsplit, jit_of(ctx), ctx->nfe_e);
  PUFE_CUDA_TRY(cudaGetLastError());
  return PUFE_OK;
}

pufe_status launch_density_fp64_bloch(pufe_ctx *ctx, const PhaseTab &ph, const double *Cr,
                                      const double *Ci, int64_t ldc, const double *f, int nocc,
                                      double *rho, cudaStream_t st) {
  auto &D = ctx->d;
  const int noccp = (nocc + 7) & ~7;
  const size_t sm = ((size_t)2 * ctx->max_basis * noccp + noccp) * sizeof(double);
  if (sm > 227 * 1024) return fail(PUFE_EINVAL, "n_e * nocc too large for the density kernel");
  auto kern = ctx->ser ? k_density_fp64<true, true> : k_density_fp64<true, false>;
  PUFE_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  kern<<<(unsigned)ctx->nelem, DEN_NT, sm, st>>>(
      D.order, D.qoff, D.xi, D.doff, D.dofs, D.ecol, D.toff, D.psi, Cr, ldc, f, nocc, noccp, rho,
      D.eshift, ph, Ci);
  PUFE_CUDA_TRY(cudaGetLastError());
  return PUFE_OK;
}

pufe_status launch_adjoint_fp64_bloch(pufe_ctx *ctx, const PhaseTab &ph, const double *Hr,
                                      const double *Hi, double *Vbar, cudaStream_t st) {
  auto &D = ctx->d;
  const int n = ctx->max_basis;
  size_t sm = (size_t)QC * n * sizeof(double) + QC * sizeof(double) + QC * sizeof(Tab1D);
  const size_t hs = (size_t)n * n * sizeof(double);
  int in_smem = (sm + hs <= 200 * 1024) ? 1 : 0;
  if (in_smem) sm += hs;
  PUFE_CUDA_TRY(cudaFuncSetAttribute(k_adjoint_fp64<true>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  k_adjoint_fp64<true><<<fp64_items(ctx), ADJ_NT, sm, st>>>(
      D.order, D.qoff, D.w, D.xi, D.doff, D.ecol, D.toff, D.psi, D.soff, D.smap, Hr, in_smem,
      Vbar, D.eshift, ph, Hi, D.wsplit, ctx->nfe_e);
  PUFE_CUDA_TRY(cudaGetLastError());
  return PUFE_OK;
}

pufe_status launch_projections(pufe_ctx *ctx, const ProjDev *pj, int P, const double *k,
                               double *F, double *Fi, cudaStream_t st) {
  auto &D = ctx->d;
  const int n = ctx->max_basis;
  const int nc = k ? 2 : 1;
  const size_t sm = ((size_t)QC * n + (size_t)nc * QC * P + (size_t)nc * n * P) * sizeof(double) +
                    QC * sizeof(Tab1D);
  if (sm > 227 * 1024) return fail(PUFE_EINVAL, "n_e * nproj too large for the projection kernel");
  if (k) {
    PUFE_CUDA_TRY(cudaFuncSetAttribute(k_projections<true>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    k_projections<true><<<(unsigned)ctx->nelem, ASM_NT, sm, st>>>(
        D.qoff, D.w, D.xi, D.x, D.doff, D.dofs, D.ecol, D.toff, D.psi, pj, P, ctx->a[0], ctx->a[1],
        ctx->a[2], F, D.eshift, phase_table(ctx, k), k[0], k[1], k[2], Fi);
  } else {
    PUFE_CUDA_TRY(cudaFuncSetAttribute(k_projections<false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    k_projections<false><<<(unsigned)ctx->nelem, ASM_NT, sm, st>>>(
        D.qoff, D.w, D.xi, D.x, D.doff, D.dofs, D.ecol, D.toff, D.psi, pj, P, ctx->a[0], ctx->a[1],
        ctx->a[2], F, nullptr, PhaseTab{}, 0.0, 0.0, 0.0, nullptr);
  }
  PUFE_CUDA_TRY(cudaGetLastError());
  return PUFE_OK;
}

}  // namespace pufe
