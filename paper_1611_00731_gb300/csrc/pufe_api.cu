// C ABI entry points of the compute calls: argument checks, device guard,
// output zeroing and dispatch to the FP64 or tensor-core kernels.
#include <cmath>
#include <vector>

#include "pufe_internal.h"

namespace pufe {
namespace {

pufe_status need_device(const pufe_ctx *ctx) {
  if (!ctx) return fail(PUFE_EINVAL, "ctx is NULL");
  if (!ctx->on_device) return fail(PUFE_ESTATE, "context was built without a CUDA device");
  return PUFE_OK;
}

struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

}  // namespace
}  // namespace pufe

using namespace pufe;

// contexts that only the FP64 kernels take: general (triclinic) cells and
// the serendipity FE space (the mixed, SCF and projector kernels are written
// for orthorhombic cells and the tricubic tensor-product space)
static bool fp64_only(const pufe_ctx *ctx) { return ctx->general || ctx->ser; }

extern "C" {

pufe_status pufe_tabulate(pufe_ctx *ctx, int prec, void *stream) {
  if (pufe_status e0 = need_device(ctx)) return e0;
  if (prec != PUFE_FP64 && prec != PUFE_TF32X3) return fail(PUFE_EINVAL, "unknown precision");
  if (prec == PUFE_TF32X3 && fp64_only(ctx))
    return fail(PUFE_EINVAL, "PUFE_TF32X3 takes orthorhombic cells with the tricubic space; general cells and the serendipity space take PUFE_FP64");
  DeviceGuard g(ctx->device);
  if (!g.ok) return fail(PUFE_ECUDA, "cudaSetDevice failed");
  pufe_status st;
  if (prec == PUFE_FP64) {
    st = launch_tabulate(ctx, (cudaStream_t)stream);
    if (st == PUFE_OK) ctx->tabulated = true;
  } else {
    st = launch_tabulate_f32(ctx, (cudaStream_t)stream);
    if (st == PUFE_OK) ctx->tabulated32 = true;
  }
  return st;
}

static pufe_status need_table(const pufe_ctx *ctx, int prec) {
  if (prec == PUFE_TF32X3 && fp64_only(ctx))
    return fail(PUFE_EINVAL, "PUFE_TF32X3 takes orthorhombic cells with the tricubic space; general cells and the serendipity space take PUFE_FP64");
  if (ctx->psi_len == 0) return PUFE_OK;
  if (prec == PUFE_FP64 && !ctx->tabulated)
    return fail(PUFE_ESTATE, "call pufe_tabulate(PUFE_FP64) first");
  if (prec == PUFE_TF32X3 && !ctx->tabulated32)
    return fail(PUFE_ESTATE, "call pufe_tabulate(PUFE_TF32X3) first");
  return PUFE_OK;
}

pufe_status pufe_assemble_HS(pufe_ctx *ctx, const double *V, int prec, int what, double *H,
                             double *S, void *stream) {
  if (pufe_status e0 = need_device(ctx)) return e0;
  if (prec != PUFE_FP64 && prec != PUFE_TF32X3) return fail(PUFE_EINVAL, "unknown precision");
  if (pufe_status e1 = need_table(ctx, prec)) return e1;
  if (what <= 0 || what > (PUFE_WANT_H | PUFE_WANT_S)) return fail(PUFE_EINVAL, "bad `what` mask");
  if ((what & PUFE_WANT_H) && (!H || !V)) return fail(PUFE_EINVAL, "H wanted: need H and V");
  if ((what & PUFE_WANT_S) && !S) return fail(PUFE_EINVAL, "S wanted: need S");
  DeviceGuard g(ctx->device);
  if (!g.ok) return fail(PUFE_ECUDA, "cudaSetDevice failed");
  cudaStream_t st = (cudaStream_t)stream;
  if (prec == PUFE_TF32X3) return launch_assemble_tc(ctx, V, what, H, S, st);
  const size_t bytes = (size_t)ctx->nnz * sizeof(double);
  if (what & PUFE_WANT_H) PUFE_CUDA_TRY(cudaMemsetAsync(H, 0, bytes, st));
  if (what & PUFE_WANT_S) PUFE_CUDA_TRY(cudaMemsetAsync(S, 0, bytes, st));
  return launch_assemble_fp64(ctx, V, what, H, S, st);
}

pufe_status pufe_assemble_HS_static(pufe_ctx *ctx, const double *V, int what, double *H,
                                    double *S, void *stream) {
  if (pufe_status e0 = need_device(ctx)) return e0;
  if (fp64_only(ctx)) return fail(PUFE_EINVAL, "pufe_assemble_HS_static takes orthorhombic cells with the tricubic space");
  if (pufe_status e1 = need_table(ctx, PUFE_TF32X3)) return e1;
  if (what <= 0 || what > (PUFE_WANT_H | PUFE_WANT_S)) return fail(PUFE_EINVAL, "bad `what` mask");
  if ((what & PUFE_WANT_H) && (!H || !V)) return fail(PUFE_EINVAL, "H wanted: need H and V");
  if ((what & PUFE_WANT_S) && !S) return fail(PUFE_EINVAL, "S wanted: need S");
  DeviceGuard g(ctx->device);
  if (!g.ok) return fail(PUFE_ECUDA, "cudaSetDevice failed");
  return launch_assemble_tc_static(ctx, V, what, H, S, (cudaStream_t)stream);
}

pufe_status pufe_density(pufe_ctx *ctx, const double *C, int64_t ldc, const double *f, int nocc,
                         int prec, double *rho, void *stream) {
  if (pufe_status e0 = need_device(ctx)) return e0;
  if (prec != PUFE_FP64 && prec != PUFE_TF32X3) return fail(PUFE_EINVAL, "unknown precision");
  if (pufe_status e1 = need_table(ctx, prec)) return e1;
  if (!C || !f || !rho) return fail(PUFE_EINVAL, "C, f and rho must not be NULL");
  if (nocc < 1 || nocc > 64 || ldc < nocc) return fail(PUFE_EINVAL, "need 1 <= nocc <= 64 and ldc >= nocc");
  DeviceGuard g(ctx->device);
  if (!g.ok) return fail(PUFE_ECUDA, "cudaSetDevice failed");
  if (prec == PUFE_FP64) return launch_density_fp64(ctx, C, ldc, f, nocc, rho, (cudaStream_t)stream);
  return launch_density_tc(ctx, C, ldc, f, nocc, rho, (cudaStream_t)stream);
}

pufe_status pufe_assemble_HV_adjoint(pufe_ctx *ctx, const double *Hbar, int prec, double *Vbar,
                                     void *stream) {
  if (pufe_status e0 = need_device(ctx)) return e0;
  if (prec != PUFE_FP64 && prec != PUFE_TF32X3) return fail(PUFE_EINVAL, "unknown precision");
  if (pufe_status e1 = need_table(ctx, prec)) return e1;
  if (!Hbar || !Vbar) return fail(PUFE_EINVAL, "Hbar and Vbar must not be NULL");
  DeviceGuard g(ctx->device);
  if (!g.ok) return fail(PUFE_ECUDA, "cudaSetDevice failed");
  if (prec == PUFE_TF32X3) return launch_adjoint_tc(ctx, Hbar, Vbar, (cudaStream_t)stream);
  return launch_adjoint_fp64(ctx, Hbar, Vbar, (cudaStream_t)stream);
}

pufe_status pufe_assemble_HS_bloch(pufe_ctx *ctx, const double *k, const double *V, int prec,
                                   int what, double *H_re, double *H_im, double *S_re,
                                   double *S_im, void *stream) {
  if (pufe_status e0 = need_device(ctx)) return e0;
  if (!k) return fail(PUFE_EINVAL, "k must not be NULL");
  if (prec != PUFE_FP64 && prec != PUFE_TF32X3) return fail(PUFE_EINVAL, "unknown precision");
  if (pufe_status e1 = need_table(ctx, prec)) return e1;
  if (what <= 0 || what > (PUFE_WANT_H | PUFE_WANT_S)) return fail(PUFE_EINVAL, "bad `what` mask");
  if ((what & PUFE_WANT_H) && (!H_re || !H_im || !V))
    return fail(PUFE_EINVAL, "H wanted: need H_re, H_im and V");
  if ((what & PUFE_WANT_S) && (!S_re || !S_im)) return fail(PUFE_EINVAL, "S wanted: need S_re, S_im");
  DeviceGuard g(ctx->device);
  if (!g.ok) return fail(PUFE_ECUDA, "cudaSetDevice failed");
  cudaStream_t st = (cudaStream_t)stream;
  if (prec == PUFE_TF32X3)
    return launch_assemble_mixed_bloch(ctx, phase_table(ctx, k), V, what, H_re, H_im, S_re, S_im,
                                       st);
  const size_t bytes = (size_t)ctx->nnz * sizeof(double);
  if (what & PUFE_WANT_H) {
    PUFE_CUDA_TRY(cudaMemsetAsync(H_re, 0, bytes, st));
    PUFE_CUDA_TRY(cudaMemsetAsync(H_im, 0, bytes, st));
  }
  if (what & PUFE_WANT_S) {
    PUFE_CUDA_TRY(cudaMemsetAsync(S_re, 0, bytes, st));
    PUFE_CUDA_TRY(cudaMemsetAsync(S_im, 0, bytes, st));
  }
  return launch_assemble_fp64_bloch(ctx, phase_table(ctx, k), V, what, H_re, H_im, S_re, S_im, st);
}

pufe_status pufe_density_bloch(pufe_ctx *ctx, const double *k, const double *C_re,
                               const double *C_im, int64_t ldc, const double *f, int nocc,
                               int prec, double *rho, void *stream) {
  if (pufe_status e0 = need_device(ctx)) return e0;
  if (prec != PUFE_FP64 && prec != PUFE_TF32X3) return fail(PUFE_EINVAL, "unknown precision");
  if (prec == PUFE_TF32X3 && fp64_only(ctx))
    return fail(PUFE_EINVAL, "PUFE_TF32X3 takes orthorhombic cells with the tricubic space; general cells and the serendipity space take PUFE_FP64");
  if (pufe_status e1 = need_table(ctx, prec)) return e1;
  if (!k || !C_re || !C_im || !f || !rho) return fail(PUFE_EINVAL, "k, C_re, C_im, f and rho must not be NULL");
  if (nocc < 1 || nocc > 64 || ldc < nocc) return fail(PUFE_EINVAL, "need 1 <= nocc <= 64 and ldc >= nocc");
  DeviceGuard g(ctx->device);
  if (!g.ok) return fail(PUFE_ECUDA, "cudaSetDevice failed");
  const PhaseTab ph = phase_table(ctx, k);
  if (prec == PUFE_TF32X3)
    return launch_density_tc(ctx, C_re, ldc, f, nocc, rho, (cudaStream_t)stream, C_im, &ph);
  return launch_density_fp64_bloch(ctx, ph, C_re, C_im, ldc, f, nocc, rho, (cudaStream_t)stream);
}

pufe_status pufe_assemble_HV_adjoint_bloch(pufe_ctx *ctx, const double *k, const double *Hbar_re,
                                           const double *Hbar_im, int prec, double *Vbar,
                                           void *stream) {
  if (pufe_status e0 = need_device(ctx)) return e0;
  if (prec != PUFE_FP64 && prec != PUFE_TF32X3) return fail(PUFE_EINVAL, "unknown precision");
  if (prec == PUFE_TF32X3 && fp64_only(ctx))
    return fail(PUFE_EINVAL, "PUFE_TF32X3 takes orthorhombic cells with the tricubic space; general cells and the serendipity space take PUFE_FP64");
  if (pufe_status e1 = need_table(ctx, prec)) return e1;
  if (!k || !Hbar_re || !Hbar_im || !Vbar) return fail(PUFE_EINVAL, "k, Hbar_re, Hbar_im and Vbar must not be NULL");
  DeviceGuard g(ctx->device);
  if (!g.ok) return fail(PUFE_ECUDA, "cudaSetDevice failed");
  const PhaseTab ph = phase_table(ctx, k);
  if (prec == PUFE_TF32X3) {
    const BlochCot bc{Hbar_im, ctx->d.eshift, ph};
    return launch_adjoint_tc(ctx, Hbar_re, Vbar, (cudaStream_t)stream, &bc);
  }
  return launch_adjoint_fp64_bloch(ctx, ph, Hbar_re, Hbar_im, Vbar, (cudaStream_t)stream);
}

// checks the projector list and copies it to the device (blocking copy)
static pufe_status upload_projectors(pufe_ctx *ctx, int nproj, const pufe_projector *proj) {
  if (nproj < 1 || nproj > 64 || !proj) return fail(PUFE_EINVAL, "need 1 <= nproj <= 64 and proj");
  std::vector<ProjDev> pd(nproj);
  for (int p = 0; p < nproj; ++p) {
    const pufe_projector &q = proj[p];
    if (q.l < 0 || q.l > 3 || q.m < -q.l || q.m > q.l || !(q.r_p > 0.0))
      return fail(PUFE_EINVAL, "projector needs 0 <= l <= 3, |m| <= l, r_p > 0");
    ProjDev d;
    for (int c = 0; c < 3; ++c) d.tau[c] = q.tau[c];
    d.l = q.l;
    d.m = q.m;
    d.rp = q.r_p;
    d.N = std::sqrt(2.0 / (std::tgamma(q.l + 1.5) * std::pow(q.r_p, 2 * q.l + 3)));
    d.rcut = q.r_p * std::sqrt(2.0 * 20.0 * std::log(10.0));   // Gaussian below 1e-20
    pd[p] = d;
  }
  if (!ctx->d.proj) PUFE_CUDA_TRY(cudaMalloc((void **)&ctx->d.proj, 64 * sizeof(ProjDev)));
  PUFE_CUDA_TRY(cudaMemcpy(ctx->d.proj, pd.data(), nproj * sizeof(ProjDev), cudaMemcpyHostToDevice));
  return PUFE_OK;
}

pufe_status pufe_nonlocal_projections(pufe_ctx *ctx, int nproj, const pufe_projector *proj,
                                      double *F, void *stream) {
  if (pufe_status e0 = need_device(ctx)) return e0;
  if (fp64_only(ctx)) return fail(PUFE_EINVAL, "this call takes orthorhombic cells with the tricubic space");
  if (pufe_status e1 = need_table(ctx, PUFE_FP64)) return e1;
  if (!F) return fail(PUFE_EINVAL, "F must not be NULL");
  DeviceGuard g(ctx->device);
  if (!g.ok) return fail(PUFE_ECUDA, "cudaSetDevice failed");
  if (pufe_status e2 = upload_projectors(ctx, nproj, proj)) return e2;
  cudaStream_t st = (cudaStream_t)stream;
  PUFE_CUDA_TRY(cudaMemsetAsync(F, 0, (size_t)ctx->n_dof * nproj * sizeof(double), st));
  return launch_projections(ctx, ctx->d.proj, nproj, nullptr, F, nullptr, st);
}

pufe_status pufe_nonlocal_projections_bloch(pufe_ctx *ctx, const double *k, int nproj,
                                            const pufe_projector *proj, double *F_re,
                                            double *F_im, void *stream) {
  if (pufe_status e0 = need_device(ctx)) return e0;
  if (fp64_only(ctx)) return fail(PUFE_EINVAL, "this call takes orthorhombic cells with the tricubic space");
  if (pufe_status e1 = need_table(ctx, PUFE_FP64)) return e1;
  if (!k || !F_re || !F_im) return fail(PUFE_EINVAL, "k, F_re and F_im must not be NULL");
  DeviceGuard g(ctx->device);
  if (!g.ok) return fail(PUFE_ECUDA, "cudaSetDevice failed");
  if (pufe_status e2 = upload_projectors(ctx, nproj, proj)) return e2;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t bytes = (size_t)ctx->n_dof * nproj * sizeof(double);
  PUFE_CUDA_TRY(cudaMemsetAsync(F_re, 0, bytes, st));
  PUFE_CUDA_TRY(cudaMemsetAsync(F_im, 0, bytes, st));
  return launch_projections(ctx, ctx->d.proj, nproj, k, F_re, F_im, st);
}

pufe_status pufe_ion_density(pufe_ctx *ctx, int natoms, const double *tau, const double *Z,
                             const double *sigma, double *rho_I, void *stream) {
  if (pufe_status e0 = need_device(ctx)) return e0;
  if (fp64_only(ctx)) return fail(PUFE_EINVAL, "this call takes orthorhombic cells with the tricubic space");
  if (natoms < 0 || !rho_I || (natoms > 0 && (!tau || !Z || !sigma)))
    return fail(PUFE_EINVAL, "need natoms >= 0, rho_I, and tau, Z, sigma for the atoms");
  for (int a = 0; a < natoms; ++a)
    if (!(sigma[a] > 0.0)) return fail(PUFE_EINVAL, "sigma must be > 0");
  DeviceGuard g(ctx->device);
  if (!g.ok) return fail(PUFE_ECUDA, "cudaSetDevice failed");
  return launch_ion_density(ctx, natoms, tau, Z, sigma, rho_I, (cudaStream_t)stream);
}

pufe_status pufe_effective_potential(pufe_ctx *ctx, const double *n, const double *rho_I,
                                     double *V_eff, double *V_C, double *eps_xc, void *stream) {
  if (pufe_status e0 = need_device(ctx)) return e0;
  if (fp64_only(ctx)) return fail(PUFE_EINVAL, "this call takes orthorhombic cells with the tricubic space");
  if (!n || !rho_I || !V_eff) return fail(PUFE_EINVAL, "n, rho_I and V_eff must not be NULL");
  DeviceGuard g(ctx->device);
  if (!g.ok) return fail(PUFE_ECUDA, "cudaSetDevice failed");
  return launch_effective_potential(ctx, n, rho_I, V_eff, V_C, eps_xc, (cudaStream_t)stream);
}

pufe_status pufe_scf_step(pufe_ctx *ctx, int nstates, const double *eps, const double *C,
                          int64_t ldc, double nelec, double kT, double alpha, int pulay, int prec,
                          const double *rho_I, const double *V_eff_in, double *n,
                          double *V_eff_out, double *f_out, pufe_scf_info *info, void *stream) {
  if (pufe_status e0 = need_device(ctx)) return e0;
  if (fp64_only(ctx)) return fail(PUFE_EINVAL, "this call takes orthorhombic cells with the tricubic space");
  if (prec != PUFE_FP64 && prec != PUFE_TF32X3) return fail(PUFE_EINVAL, "unknown precision");
  if (pufe_status e1 = need_table(ctx, prec)) return e1;
  if (nstates < 1 || nstates > 64 || ldc < nstates)
    return fail(PUFE_EINVAL, "need 1 <= nstates <= 64 and ldc >= nstates");
  if (!eps || !C || !rho_I || !V_eff_in || !n || !V_eff_out)
    return fail(PUFE_EINVAL, "eps, C, rho_I, V_eff_in, n and V_eff_out must not be NULL");
  if (!(kT > 0.0) || !(nelec > 0.0) || nelec > 2.0 * nstates)
    return fail(PUFE_EINVAL, "need kT > 0 and 0 < nelec <= 2 nstates");
  if (!ctx->scf) return fail(PUFE_ESTATE, "call pufe_ion_density first");
  if (pulay < 0 || pulay > 8) return fail(PUFE_EINVAL, "need 0 <= pulay <= 8");
  DeviceGuard g(ctx->device);
  if (!g.ok) return fail(PUFE_ECUDA, "cudaSetDevice failed");
  return launch_scf_step(ctx, nstates, eps, C, ldc, nelec, kT, alpha, pulay, prec, rho_I, V_eff_in, n,
                         V_eff_out, f_out, info, (cudaStream_t)stream);
}

pufe_status pufe_scf_step_bloch(pufe_ctx *ctx, int nk, const double *kpts, const double *wk,
                                int nstates, const double *eps, const double *const *C_re,
                                const double *const *C_im, int64_t ldc, double nelec, double kT,
                                double alpha, int pulay, int prec, const double *rho_I,
                                const double *V_eff_in, double *n, double *V_eff_out,
                                double *f_out, pufe_scf_info *info, void *stream) {
  if (pufe_status e0 = need_device(ctx)) return e0;
  if (fp64_only(ctx)) return fail(PUFE_EINVAL, "this call takes orthorhombic cells with the tricubic space");
  if (prec != PUFE_FP64 && prec != PUFE_TF32X3) return fail(PUFE_EINVAL, "unknown precision");
  if (pufe_status e1 = need_table(ctx, prec)) return e1;
  if (nk < 1 || nk > 64) return fail(PUFE_EINVAL, "need 1 <= nk <= 64");
  if (nstates < 1 || nstates > 64 || ldc < nstates)
    return fail(PUFE_EINVAL, "need 1 <= nstates <= 64 and ldc >= nstates");
  if (!kpts || !wk || !eps || !C_re || !C_im || !rho_I || !V_eff_in || !n || !V_eff_out)
    return fail(PUFE_EINVAL,
                "kpts, wk, eps, C_re, C_im, rho_I, V_eff_in, n and V_eff_out must not be NULL");
  double wsum = 0.0;
  for (int i = 0; i < nk; ++i) {
    if (!(wk[i] > 0.0)) return fail(PUFE_EINVAL, "k-point weights must be > 0");
    if (!C_re[i] || !C_im[i]) return fail(PUFE_EINVAL, "an eigenvector array is NULL");
    wsum += wk[i];
  }
  if (std::fabs(wsum - 1.0) > 1e-12) return fail(PUFE_EINVAL, "k-point weights must sum to 1");
  if (!(kT > 0.0) || !(nelec > 0.0) || nelec > 2.0 * nstates)
    return fail(PUFE_EINVAL, "need kT > 0 and 0 < nelec <= 2 nstates");
  if (!ctx->scf) return fail(PUFE_ESTATE, "call pufe_ion_density first");
  if (pulay < 0 || pulay > 8) return fail(PUFE_EINVAL, "need 0 <= pulay <= 8");
  DeviceGuard g(ctx->device);
  if (!g.ok) return fail(PUFE_ECUDA, "cudaSetDevice failed");
  return launch_scf_step_bloch(ctx, nk, kpts, wk, nstates, eps, C_re, C_im, ldc, nelec, kT, alpha,
                               pulay, prec, rho_I, V_eff_in, n, V_eff_out, f_out, info,
                               (cudaStream_t)stream);
}

pufe_status pufe_scf_reset(pufe_ctx *ctx) {
  if (pufe_status e0 = need_device(ctx)) return e0;
  scf_reset(ctx);
  return PUFE_OK;
}

pufe_status pufe_autotune(pufe_ctx *ctx, int *nclasses, void *stream) {
  if (pufe_status e0 = need_device(ctx)) return e0;
  if (fp64_only(ctx)) return fail(PUFE_EINVAL, "the mixed path takes orthorhombic cells with the tricubic space");
  DeviceGuard g(ctx->device);
  if (!g.ok) return fail(PUFE_ECUDA, "cudaSetDevice failed");
  return autotune_strip(ctx, nclasses, (cudaStream_t)stream);
}

pufe_status pufe_selftest_timeout(pufe_ctx *ctx, uint64_t wait_ns, void *stream) {
  if (pufe_status e0 = need_device(ctx)) return e0;
  if (wait_ns < 1000000ull || wait_ns > 2000000000ull)
    return fail(PUFE_EINVAL, "wait_ns must be between 1e6 and 2e9");
  DeviceGuard g(ctx->device);
  if (!g.ok) return fail(PUFE_ECUDA, "cudaSetDevice failed");
  return launch_wait_probe(ctx, wait_ns, (cudaStream_t)stream);
}

pufe_status pufe_profile_assembly(pufe_ctx *ctx, int enable) {
  if (pufe_status e0 = need_device(ctx)) return e0;
  DeviceGuard g(ctx->device);
  if (!g.ok) return fail(PUFE_ECUDA, "cudaSetDevice failed");
  return profile_enable(ctx, enable != 0);
}

pufe_status pufe_profile_read(pufe_ctx *ctx, double *ms) {
  if (pufe_status e0 = need_device(ctx)) return e0;
  if (!ms) return fail(PUFE_EINVAL, "ms must not be NULL");
  DeviceGuard g(ctx->device);
  if (!g.ok) return fail(PUFE_ECUDA, "cudaSetDevice failed");
  return profile_read(ctx, ms);
}

pufe_status pufe_sync_status(pufe_ctx *ctx, void *stream) {
  if (pufe_status e0 = need_device(ctx)) return e0;
  DeviceGuard g(ctx->device);
  if (!g.ok) return fail(PUFE_ECUDA, "cudaSetDevice failed");
  PUFE_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
  unsigned flag = 0;
  PUFE_CUDA_TRY(cudaMemcpy(&flag, ctx->d.err, sizeof(unsigned), cudaMemcpyDeviceToHost));
  if (flag) {
    PUFE_CUDA_TRY(cudaMemset(ctx->d.err, 0, sizeof(unsigned)));
    if (flag & DEVERR_TIMEOUT) return fail(PUFE_ETIMEOUT, "a device wait gave up");
    if (flag == DEVERR_NONFINITE)
      return fail(PUFE_EINVAL, "V holds a NaN or an infinity (the assembly read it)");
    return fail(PUFE_EDEVICE, "kernel reported device error flag " + std::to_string(flag));
  }
  return PUFE_OK;
}

}  // extern "C"
