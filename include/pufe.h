/*
 * pufe.h -- C ABI of the GB300 PUFE hot path.
 *
 * The library assembles the partition-of-unity finite element (PUFE)
 * Hamiltonian H and overlap S of a periodic cell at the Gamma point, and
 * evaluates the electron density at the quadrature points, on one NVIDIA
 * GB300 (sm_103a).  It follows Pask & Sukumar, "Partition of unity finite
 * element method for quantum mechanical materials calculations":
 *   - basis (Sec. 4, eqs. pufebasis/psih): tricubic Lagrange FE functions on
 *     every node, plus trilinear-PU x enrichment products phi_j^PU Psi_alpha
 *     on every PU vertex j within r_e of alpha's atom (Sec. 5.1);
 *   - enrichments (Sec. 5.1, eqs. Psitilde/Psi): R_nl(r) Y_lm h(r, r_c),
 *     summed over periodic images; R_nl is a normalised Slater-type orbital
 *     N r^(n-1) e^(-zeta r), Y_lm real and unit-normalised;
 *   - matrices (Sec. 4, eq. disceig3d, local potential):
 *       H_ij = int 1/2 grad phi_i . grad phi_j + phi_i V phi_j,
 *       S_ij = int phi_i phi_j,
 *     with every integral taken on one shared element quadrature rule
 *     (Sec. 5.2);
 *   - density (Sec. 3, eq. rhoe): n(x_q) = sum_k f_k |psi_k(x_q)|^2 >= 0
 *     (the paper's rho_e = -n).
 *
 * Conventions
 *   Units: bohr and hartree.  Orthorhombic cells, or general (triclinic)
 *   cells given by their lattice vectors (pufe_cell.lattice).
 *   Numbering: elements e = ex + nx (ey + ny ez).  FE DOFs are the nodes of
 *   the (3nx)(3ny)(3nz) periodic grid, index gx + 3nx (gy + 3ny gz) (the
 *   serendipity space keeps the vertex and edge nodes, renumbered in that
 *   order); they are followed by the enrichment DOFs ordered by (atom,
 *   orbital, enriched vertex index).  Quadrature points are stored element by element; within
 *   an element a tensor rule runs x fastest, and subdivided cells are
 *   visited depth first in the order a + 2b + 4c of their octant offsets.
 *   Matrices: one CSR pattern (int64 row pointers, int32 sorted column
 *   indices, both triangles stored) shared by H and S; values are float64.
 *   Ownership: the caller owns every pointer it passes.  The context owns
 *   the mesh, rules, tables and work arrays and frees them in
 *   pufe_destroy.  Device pointers must be on the context's device.
 *   Streams: `stream` is a cudaStream_t (NULL = legacy default stream).
 *   Compute calls are asynchronous on that stream; they never synchronise.
 *   The mixed-precision assembly forks part of its work onto a stream the
 *   context owns and joins it back into `stream` before returning, so its
 *   results are ordered on `stream` like any other call.  Issue the calls on
 *   one context from one host thread at a time.
 *   Errors: every call returns a pufe_status; pufe_last_error() gives a
 *   message for the calling thread.  No call aborts or throws.
 */
#ifndef PUFE_H
#define PUFE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pufe_ctx pufe_ctx;

typedef enum {
  PUFE_OK = 0,
  PUFE_EINVAL = 1,   /* bad argument (size, pointer, mode) */
  PUFE_ENOMEM = 2,   /* host or device allocation failed */
  PUFE_ECUDA = 3,    /* a CUDA runtime call failed */
  PUFE_ENOTSPD = 4,  /* reserved: S not positive definite */
  PUFE_ENOTCONV = 5, /* reserved: SCF did not converge */
  PUFE_ETIMEOUT = 6, /* a bounded device wait gave up */
  PUFE_EDEVICE = 7,  /* a kernel reported a device-side error flag */
  PUFE_ESTATE = 8    /* call out of order (e.g. assemble before tabulate) */
} pufe_status;

/* Arithmetic of the element contractions. */
typedef enum {
  PUFE_FP64 = 0,   /* FP64 everywhere (plain CUDA cores) */
  PUFE_TF32X3 = 1  /* mixed precision: element contractions in FP32 with
                      FP64 global accumulation.  Elements with n_e <= 128
                      run on the CUDA cores (FP32 FMA, round to nearest),
                      the FE-FE V block and the FE-enrichment blocks by sum
                      factorization over the tensor-product rule; elements
                      with 128 < n_e <= 256 run their enrichment strip on
                      the tensor cores (tcgen05 kind::tf32, every operand
                      split into two TF32 terms, hi*hi + hi*lo + lo*hi).
                      The constant FE-FE blocks of T and S are exact FP64
                      constants, and the enrichment-enrichment block of S
                      (ill-conditioned, Sec. 6.2 Table 1) is computed in
                      FP64 arithmetic from the FP32 enrichment values.  FP32
                      tabulation, density and adjoint. */
} pufe_prec;

/* Quadrature modes (Sec. 5.2). */
enum {
  PUFE_QUAD_FIXED = 0,  /* p_near^3 Gauss on elements within r_c of an atom
                           image, p_far^3 elsewhere */
  PUFE_QUAD_PADAPT = 1, /* per element the smallest p in [p_min, p_max] with
                           |I_p - I_(p+2)| < tol for Psi^2 and |grad Psi|^2 of
                           every enrichment of the element; p_min^3 on
                           elements without enrichment */
  PUFE_QUAD_HADAPT = 2  /* the paper's recursive scheme: 5^3 against the 8^3
                           reference, failing integrands passed to the 8
                           children, 8^3 kept on accepted (or max_depth)
                           cells; p_far^3 on elements without enrichment */
};

/* what to assemble */
enum { PUFE_WANT_H = 1, PUFE_WANT_S = 2 };

/* Classical FE part of the basis (Sec. 4; Sec. 6 uses the serendipity one). */
enum {
  PUFE_FE_LAGRANGE64 = 0,   /* tricubic Lagrange hexahedra, 64 nodes per element */
  PUFE_FE_SERENDIPITY32 = 1 /* cubic serendipity hexahedra, 32 nodes per element: the
                               vertices and two inner nodes per edge of the
                               tricubic grid, numbered compactly in grid order;
                               element columns in ascending local-node order.
                               Tabulation, assembly (Gamma and Bloch), density
                               and adjoint in PUFE_FP64; the other calls
                               return PUFE_EINVAL */
};

typedef struct {
  double a[3];         /* cell edge lengths (bohr) of an orthorhombic cell */
  int nel[3];          /* elements per axis, each >= 1 */
  int natoms;          /* >= 0 */
  const double *tau;   /* natoms x 3 Cartesian positions (host) */
  const int *species;  /* natoms species indices (host) */
  const double *lattice; /* NULL: the orthorhombic cell a[].  Else a general
                            (triclinic) cell (Sec. 6.2, the CeAl cell): 9
                            values (host), the rows a_1, a_2, a_3 in bohr,
                            divided into nel[d] elements along a_d; each
                            element is a parallelepiped x = x_0 + J (xi + 1),
                            J = [a_1/2nel_1, a_2/2nel_2, a_3/2nel_3], and a[]
                            is not read.  General cells take the FP64 path
                            (tabulation, assembly, Bloch assembly, density,
                            adjoint); the other calls return PUFE_EINVAL. */
  int fe_space;        /* PUFE_FE_LAGRANGE64 (0) or PUFE_FE_SERENDIPITY32 */
} pufe_cell;

typedef struct {
  int norb;            /* enrichment orbitals of this species, >= 0 */
  const int *n;        /* principal quantum numbers, 1 <= n <= 8 (host) */
  const int *l;        /* 0 <= l <= 3, l < n (host) */
  const int *m;        /* -l <= m <= l (host) */
  const double *zeta;  /* Slater exponents > 0 (host) */
  double r_c;          /* cutoff radius of h(r, r_c) (bohr), > 0 */
  double r_e;          /* support radius: vertices within r_e are enriched */
} pufe_species;

typedef struct {
  int mode;            /* PUFE_QUAD_* */
  int p_far, p_near;   /* FIXED: Gauss orders; HADAPT: p_far for plain cells */
  int p_min, p_max;    /* PADAPT range (1..16) */
  double tol;          /* absolute tolerance of the adaptive tests */
  int max_depth;       /* HADAPT subdivision depth limit (0..4) */
  int device_tests;    /* PADAPT / HADAPT: 0 evaluates the tests' integrals
                          on the host cores, 1 on the current CUDA device
                          (one CTA per test, every test of an order set or
                          subdivision level in one launch; PUFE_ECUDA
                          without a device).  The decisions, points and
                          point order are those of the host construction;
                          only the summation order of the integrals
                          differs (a test within rounding of tol may
                          decide the other way). */
} pufe_quad;

/* Build the mesh, enrichment sets, quadrature rules, CSR pattern and scatter
 * maps on the host (Secs. 4, 5.1, 5.2) and copy them to the current CUDA
 * device.  Blocking.  *out receives a new context. */
pufe_status pufe_build_mesh(const pufe_cell *cell, const pufe_species *species,
                            int nspecies, const pufe_quad *quad, pufe_ctx **out);

/* Sizes: number of DOFs N, CSR non-zeros, quadrature points, elements and
 * the largest element basis size.  Any pointer may be NULL. */
pufe_status pufe_get_sizes(const pufe_ctx *ctx, int64_t *n_dof, int64_t *nnz,
                           int64_t *n_q, int64_t *n_elem, int64_t *max_basis);

/* Copy the quadrature rule to host buffers: points x (n_q x 3), weights w
 * (n_q, Jacobian folded in) and element offsets (n_elem + 1).  NULL skips. */
pufe_status pufe_get_quadrature(const pufe_ctx *ctx, double *x, double *w,
                                int64_t *elem_offsets);

/* Copy the CSR pattern to host buffers rowptr (N + 1) and col (nnz). */
pufe_status pufe_get_pattern(const pufe_ctx *ctx, int64_t *rowptr, int32_t *col);

/* Per-element basis sizes n_e (n_elem int32, host) and, optionally, the
 * global DOF of every element column (sum n_e int32, host; element-major,
 * 64 FE columns first). */
pufe_status pufe_get_element_basis(const pufe_ctx *ctx, int32_t *n_e, int32_t *dofs);

/* K0 (Sec. 5.1, eqs. Psitilde/Psi): tabulate Psi_alpha and grad Psi_alpha at
 * every quadrature point of every element for the enrichments that appear in
 * that element's basis.  The table lives in the context and is read by the
 * assembly, density and adjoint kernels of the same precision: `prec` =
 * PUFE_FP64 fills the FP64 table, PUFE_TF32X3 the FP32 table.  Asynchronous
 * on `stream`. */
pufe_status pufe_tabulate(pufe_ctx *ctx, int prec, void *stream);

/* K1-K3 (Sec. 4, eq. disceig3d): H and/or S values into caller-owned device
 * arrays of nnz float64 each (pattern of pufe_get_pattern).  V (n_q float64,
 * device) is the local potential at the quadrature points; it may be NULL
 * when only S is wanted.  The arrays are overwritten.  `what` is a mask of
 * PUFE_WANT_H | PUFE_WANT_S.  Requires a prior pufe_tabulate of the same
 * precision.  PUFE_TF32X3 additionally needs every (sub)cell rule to have
 * between 4 points per axis (so that the FE-FE blocks of T and S are exact
 * constants) and 16, and n_e <= 256; otherwise it returns PUFE_EINVAL.
 * Asynchronous. */
pufe_status pufe_assemble_HS(pufe_ctx *ctx, const double *V, int prec, int what,
                             double *H, double *S, void *stream);

/* Allocation-free variant of pufe_assemble_HS with prec = PUFE_TF32X3 (the
 * paper has no counterpart; it exists for callers).  Some callers cannot
 * allocate device memory while they run their solve loop -- for example code
 * that must stay inside a fixed device-memory budget, or that runs where the
 * allocator may not be called.  This call allocates nothing: the FP32 copy of
 * V that the tensor-core assembly reads (elements with n_e > 128) lives in a
 * library-owned static device array of PUFE_STATIC_MAX_POINTS (4,194,304)
 * floats, resident on
 * every device that loads the library until the process exits.  The array
 * holds V on the padded points of the n_e > 128 elements only: contexts whose
 * last such element ends beyond PUFE_STATIC_MAX_POINTS padded points return
 * PUFE_EINVAL (contexts without such elements never touch it).  The
 * context itself (built earlier by pufe_build_mesh) and a prior
 * pufe_tabulate(ctx, PUFE_TF32X3) are still required; arguments and results
 * are as for pufe_assemble_HS.  The first call on a device looks up the
 * array's device address, so make that first call before capturing the
 * stream; the address is kept for the life of the device's primary context
 * (after a cudaDeviceReset the process must not call this entry point
 * again).  All calls share the one array: each call rewrites the entries it
 * reads, and calls that overlap on the GPU (on different streams or
 * contexts) race on it.  Asynchronous. */
pufe_status pufe_assemble_HS_static(pufe_ctx *ctx, const double *V, int what, double *H,
                                    double *S, void *stream);

/* K4 (Sec. 3, eq. rhoe): n_q = sum_k f_k (sum_j B_qj C_jk)^2 for every
 * quadrature point.  C: device float64, N x nocc, row-major with leading
 * dimension ldc >= nocc (C[j * ldc + k]); f: device float64 (nocc);
 * rho: device float64 (n_q), overwritten.  1 <= nocc <= 64.  PUFE_TF32X3
 * evaluates in FP32 on the CUDA cores.  Asynchronous. */
pufe_status pufe_density(pufe_ctx *ctx, const double *C, int64_t ldc,
                         const double *f, int nocc, int prec, double *rho,
                         void *stream);

/* K5, adjoint of V -> H (Sec. 4): Vbar_q = w_q b_q^T Hbar_e b_q for a
 * cotangent Hbar given as nnz float64 values on the CSR pattern (device).
 * Vbar: device float64 (n_q), overwritten.  With Hbar = sum_k f_k c_k c_k^T
 * this equals w_q n_q.  PUFE_TF32X3 evaluates in FP32.  Asynchronous. */
pufe_status pufe_assemble_HV_adjoint(pufe_ctx *ctx, const double *Hbar, int prec, double *Vbar,
                                     void *stream);

/* ---- Bloch-periodic states, k != 0 (Sec. 4, eqs. bloch, strong) --------- */

/* H(k) and/or S(k) of the Bloch-periodic basis at wavevector k (host,
 * 3 components, 1/bohr): the same element matrices as pufe_assemble_HS,
 * scattered with the phase exp(i k.(R_j - R_i)) of each column pair, where
 * R_i is the lattice translation that maps the column's node or PU vertex
 * onto its representative in the cell (the enrichments themselves are
 * periodic, Sec. 5.1 eq. Psi with f(R) = 1).  Outputs are the real and
 * imaginary parts, each nnz float64 on the CSR pattern (device,
 * overwritten; H(k) and S(k) are Hermitian).  prec PUFE_FP64 needs
 * pufe_tabulate(ctx, PUFE_FP64); PUFE_TF32X3 (meshes with n_e <= 128) the
 * PUFE_TF32X3 table and rules of >= 4 points per axis: the element blocks of
 * the mixed pufe_assemble_HS, the FE-FE blocks (with the exact kinetic and
 * overlap constants) scattered with FP64 phases and the enrichment blocks with
 * FP32 phases.  k = 0 gives the Gamma-point matrices with zero imaginary
 * parts.  Asynchronous. */
pufe_status pufe_assemble_HS_bloch(pufe_ctx *ctx, const double *k, const double *V, int prec,
                                   int what, double *H_re, double *H_im, double *S_re,
                                   double *S_im, void *stream);

/* Density of complex Bloch states: n_q = sum_j f_j |sum_l B_ql
 * exp(i k.R_l) C_lj|^2 with C = C_re + i C_im (device float64, N x nocc, row
 * stride ldc).  Other arguments as pufe_density: PUFE_FP64 (any cell) or
 * PUFE_TF32X3 (orthorhombic cells: the phased coefficients formed in FP64,
 * rounded to FP32, real and imaginary parts summed in FP32 on the CUDA
 * cores).  Asynchronous. */
pufe_status pufe_density_bloch(pufe_ctx *ctx, const double *k, const double *C_re,
                               const double *C_im, int64_t ldc, const double *f, int nocc,
                               int prec, double *rho, void *stream);

/* Adjoint of V -> H(k) for a complex cotangent Hbar = Hbar_re + i Hbar_im
 * (device, nnz each): Vbar_q = w_q Re sum_ij conj(Hbar[g_i, g_j])
 * exp(i k.(R_j - R_i)) b_i b_j, the derivative of Re sum conj(Hbar) H(k).
 * PUFE_FP64 (any cell) or PUFE_TF32X3 (orthorhombic cells: the phased real
 * element block formed in FP64 from the two CSR values, then the kernels of
 * pufe_assemble_HV_adjoint in FP32).  Asynchronous. */
pufe_status pufe_assemble_HV_adjoint_bloch(pufe_ctx *ctx, const double *k, const double *Hbar_re,
                                           const double *Hbar_im, int prec, double *Vbar,
                                           void *stream);

/* ---- separable nonlocal projectors (Sec. 4, eq. disceig3d) -------------- */

/* A Gaussian projector v(x) = N r^l exp(-r^2 / (2 r_p^2)) Y_lm(r_hat),
 * r = |x - tau - R| summed over lattice translations R, with
 * N = sqrt(2 / (Gamma(l + 3/2) r_p^(2l+3))) so that int v^2 = 1 (the paper's
 * projectors come from pseudopotential tables not used here). */
typedef struct {
  double tau[3];  /* centre (bohr) */
  int l, m;       /* 0 <= l <= 3, -l <= m <= l (real Y_lm, as the enrichments) */
  double r_p;     /* width (bohr), > 0 */
} pufe_projector;

/* Projections F[i, p] = int phi_i v_p of every basis function onto nproj
 * projectors (1 <= nproj <= 64; host array), on the shared element rule, at
 * the Gamma point: the nonlocal term of H is F h F^T for the caller's
 * projector weights h (a rank-nproj update that may fill entries outside the
 * sparse pattern, so it is returned as F).  F: device float64, N x nproj
 * row-major (F[i * nproj + p]), overwritten.  Needs pufe_tabulate(ctx,
 * PUFE_FP64).  Asynchronous apart from a blocking copy of the projector
 * list. */
pufe_status pufe_nonlocal_projections(pufe_ctx *ctx, int nproj, const pufe_projector *proj,
                                      double *F, void *stream);

/* The same projections at wavevector k (host array of 3, 1/bohr; Sec. 4,
 * eqs. bloch, strong): the projector is the Bloch sum
 * p^k(x) = sum_n exp(i k.a_n) v(x - tau - a_n) and the basis functions are the
 * Bloch sums of pufe_assemble_HS_bloch, so
 * F[g, p] = int conj(phi_g^k) p^k, returned as F_re + i F_im (device float64,
 * N x nproj row-major each, overwritten); the nonlocal term of H(k) is
 * F h F^H.  k = 0 gives F_im = 0 and F_re = pufe_nonlocal_projections.
 * Needs pufe_tabulate(ctx, PUFE_FP64).  Asynchronous apart from a blocking
 * copy of the projector list. */
pufe_status pufe_nonlocal_projections_bloch(pufe_ctx *ctx, const double *k, int nproj,
                                            const pufe_projector *proj, double *F_re,
                                            double *F_im, void *stream);

/* ---- self-consistent field (Sec. 3) ------------------------------------ */

/* Ionic charge density at every quadrature point (Sec. 3: the ionic
 * potentials are generated by localized ionic charges): Gaussian charges
 * Z_a exp(-r^2/sigma_a^2) / (pi^(3/2) sigma_a^3) of natoms atoms summed over
 * periodic images.  tau: natoms x 3 Cartesian positions, Z, sigma: natoms
 * values (host).  rho_I: device float64 (n_q), overwritten.  The context
 * keeps sum_a Z_a^2 / (sigma_a sqrt(2 pi)), the Gaussians' self-energy, for
 * pufe_scf_step.  The first SCF call of a context allocates its work arrays
 * (a few n_q and N_fe float64 vectors).  Asynchronous apart from a blocking
 * copy of the atom list. */
pufe_status pufe_ion_density(pufe_ctx *ctx, int natoms, const double *tau, const double *Z,
                             const double *sigma, double *rho_I, void *stream);

/* Effective potential V_eff = V_C + v_xc at the quadrature points (Sec. 3,
 * eqs. veff, poisson).  V_C is the total Coulomb potential of the charge
 * rho = rho_I - n, from del^2 V_C = 4 pi rho in the tricubic FE space of the
 * mesh (weak form on the shared element rule, zero cell average; the charge
 * must be neutral); v_xc is the LDA (Dirac exchange with the Perdew-Zunger
 * 1981 correlation, unpolarised).  n, rho_I: device float64 (n_q); V_eff:
 * device float64 (n_q), overwritten; V_C and eps_xc (the LDA energy per
 * electron) are optional outputs (NULL skips).  FP64.  Asynchronous. */
pufe_status pufe_effective_potential(pufe_ctx *ctx, const double *n, const double *rho_I,
                                     double *V_eff, double *V_C, double *eps_xc, void *stream);

/* Energies of one SCF step (hartree) and its density residual. */
typedef struct {
  double mu;        /* Fermi level of the occupations */
  double e_band;    /* sum_k f_k eps_k */
  double e_dc;      /* -int n_out V_eff,in */
  double e_es;      /* -1/2 int (rho_I - n_out) V_C[n_out] */
  double e_self;    /* self-energy of the Gaussian ions (subtracted) */
  double e_xc;      /* int n_out eps_xc(n_out) */
  double e_ts;      /* -kT S of the occupations */
  double e_total;   /* e_band + e_dc + e_es - e_self + e_xc + e_ts */
  double residual;  /* int |n_out - n_in| */
} pufe_scf_info;

/* One fixed-point step of the SCF iteration (Sec. 3, fig. scf) after the
 * caller's eigensolve of H[V_eff,in] c = eps S c (assembled with
 * pufe_assemble_HS).  eps: nstates eigenvalues (host, 1 <= nstates <= 64);
 * C: device float64 eigenvectors, N x nstates with leading dimension ldc,
 * S-orthonormal.  Occupations f_k = 2 / (1 + exp((eps_k - mu)/kT)) with
 * sum f = nelec (kT > 0); the output density n_out = sum f |psi|^2 (through
 * pufe_density with `prec`); energies of n_out (pufe_scf_info); density
 * mixing in place (n: device float64, n_q, the input density on entry):
 * pulay <= 1: linear, n <- n + alpha (n_out - n); 2 <= pulay <= 8: Pulay
 * (DIIS) over the last `pulay` steps of this context (input densities and
 * residuals R = n_out - n kept in the context, cleared by pufe_scf_reset):
 * n <- sum_i c_i (n_i + alpha R_i) with sum c_i = 1 minimising
 * || sum_i c_i R_i || in the quadrature-weighted norm.  V_eff_out =
 * V_eff[n] of the mixed density.
 * rho_I, V_eff_in: device float64 (n_q).  f_out (host, nstates) and info may
 * be NULL.  Needs a prior pufe_ion_density and pufe_tabulate(prec).
 * Blocking: returns after the step has finished on `stream`. */
pufe_status pufe_scf_step(pufe_ctx *ctx, int nstates, const double *eps, const double *C,
                          int64_t ldc, double nelec, double kT, double alpha, int pulay, int prec,
                          const double *rho_I, const double *V_eff_in, double *n,
                          double *V_eff_out, double *f_out, pufe_scf_info *info, void *stream);

/* One SCF step with k-point sampling (Sec. 4, eqs. bloch, strong; Sec. 3),
 * after the caller's eigensolves of H(k) c = eps S(k) c (pufe_assemble_HS_bloch)
 * at nk wavevectors kpts (host, nk x 3, 1/bohr) with weights wk (host, nk,
 * each > 0, summing to 1; a time-reversal pair k, -k is one point of twice
 * the weight): eps (host, nk x nstates, k-major) and the S(k)-orthonormal
 * eigenvectors C_re[i] + i C_im[i] (host arrays of nk device pointers, each
 * N x nstates float64 with leading dimension ldc).  One Fermi level for all k:
 * f_nk = 2 / (1 + exp((eps_nk - mu)/kT)) with sum_k w_k sum_n f_nk = nelec;
 * n_out = sum_k w_k sum_n f_nk |psi_nk|^2 (pufe_density_bloch with `prec`);
 * e_band = sum_k w_k sum_n f_nk eps_nk and the entropy term weighted alike;
 * energies, mixing (the same Pulay history) and the new potential as
 * pufe_scf_step.  1 <= nk <= 64; f_out (host, nk x nstates) may be NULL.
 * Blocking: returns after the step has finished on `stream`. */
pufe_status pufe_scf_step_bloch(pufe_ctx *ctx, int nk, const double *kpts, const double *wk,
                                int nstates, const double *eps, const double *const *C_re,
                                const double *const *C_im, int64_t ldc, double nelec, double kT,
                                double alpha, int pulay, int prec, const double *rho_I,
                                const double *V_eff_in, double *n, double *V_eff_out,
                                double *f_out, pufe_scf_info *info, void *stream);

/* Forget the Pulay history of the context (start of a new SCF run). */
pufe_status pufe_scf_reset(pufe_ctx *ctx);

/* Number of enrichment functions (slots) in each element's basis: n_elem
 * int32 (host).  An element's enrichment columns are its slots times their
 * enriched vertices; its K0 table holds 4 values per slot and point. */
pufe_status pufe_get_element_slots(const pufe_ctx *ctx, int32_t *n_slot);

/* Autotuner of the mixed assembly (the batching of the element classes; the
 * paper prescribes no kernel).  The enrichment strip forms the
 * enrichment-enrichment block of H either from slot-pair projections or from
 * direct 4 x 4 tiles; by default each element takes the form with the lower
 * operation count.  This call groups the strip elements (64 < n_e <= 128, at
 * most 8 enrichments) into classes of equal n_e, enrichment count and
 * (sub)cell rules, times both forms on the GPU on each class (up to 256 of
 * its elements, best of 3 after a warm-up), and keeps the faster one for
 * every element of the class.  If the environment variable
 * PUFE_AUTOTUNE_CACHE names a file, classes listed there (a line "key form",
 * form 1 = slot pairs, 2 = tiles) are taken without timing and new decisions
 * are appended.  *nclasses (may be NULL) receives the number of classes set.
 * Needs pufe_tabulate(ctx, PUFE_TF32X3); allocates and frees scratch (H, S
 * and V sized arrays); blocking; results of later assemblies are unchanged
 * up to the forms' FP32 rounding.  Orthorhombic cells only. */
pufe_status pufe_autotune(pufe_ctx *ctx, int *nclasses, void *stream);

/* ---- diagnostics and instrumentation (no counterpart in the paper) ------- */

/* Exercise the timeout path of the device waits: one thread waits, with the
 * same bounded mbarrier wait the pipelined tensor-core kernels use, on a
 * barrier that nothing completes; after wait_ns nanoseconds (1e6 <= wait_ns
 * <= 2e9) it gives up, sets the context's device error flag and returns, so
 * the next pufe_sync_status reports PUFE_ETIMEOUT (and clears the flag) and
 * the context stays usable.  Asynchronous on `stream`. */
pufe_status pufe_selftest_timeout(pufe_ctx *ctx, uint64_t wait_ns, void *stream);


/* enable != 0: the following pufe_assemble_HS calls with PUFE_TF32X3 record
 * CUDA events around each of their kernels, on the stream each kernel runs
 * on (the first enable creates the events); enable = 0 stops it.  Results
 * are unchanged.  Not for calls inside a CUDA graph capture. */
pufe_status pufe_profile_assembly(pufe_ctx *ctx, int enable);

/* Durations in ms of the last instrumented assembly call, ms[5] (host):
 * [0] the whole call, [1] the FE-FE kernel (kinetic constants and the V
 * block), [2] the enrichment-enrichment kernel of S, [3] the tensor-core tile
 * kernel, [4] the enrichment strip kernel; 0 for a kernel the call did not
 * launch.  Kernels on the two streams overlap, so the parts need not add up
 * to the whole.  Waits for the call to finish.  PUFE_ESTATE if no
 * instrumented call was made. */
pufe_status pufe_profile_read(pufe_ctx *ctx, double *ms);

/* Wait for `stream`, then report (and clear) any device-side error flag:
 * PUFE_ETIMEOUT for a bounded wait that gave up, PUFE_EINVAL when an
 * assembly read a NaN or infinite V, PUFE_EDEVICE for any other flag. */
pufe_status pufe_sync_status(pufe_ctx *ctx, void *stream);

/* Release the context and everything it owns.  NULL is a no-op. */
void pufe_destroy(pufe_ctx *ctx);

/* Message of the last failing call on this thread ("" if none). */
const char *pufe_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* PUFE_H */
