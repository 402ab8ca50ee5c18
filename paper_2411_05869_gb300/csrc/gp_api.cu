// gp_api.cu -- the C-ABI of libgp.so (declared in include/gp.h): handle management, argument checks,
// device memory accounting and the calls into the step implementations.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>

#include "gp_internal.cuh"

// ------------------------------------------------------------------------------------------ memory
void* dev_alloc(gp_ctx* ctx, std::vector<DevBuf>& owner, size_t bytes) {
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) & ~size_t(255);
  if (ctx->budget && ctx->held.load() + bytes > ctx->budget)
    throw GpError{GP_ERR_NOMEM, "device memory budget exceeded (" + std::to_string(ctx->held.load() + bytes) +
                                    " > " + std::to_string(ctx->budget) + " bytes)"};
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw GpError{GP_ERR_NOMEM, std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e)};
  }
  owner.push_back(DevBuf{p, bytes});
  ctx->held += bytes;
  return p;
}

void dev_free_all(gp_ctx* ctx, std::vector<DevBuf>& owner) {
  if (!owner.empty()) cudaStreamSynchronize(ctx->stream);
  for (auto& b : owner) {
    cudaFree(b.p);
    ctx->held.fetch_sub(std::min(ctx->held.load(), b.bytes));
  }
  owner.clear();
}

namespace {

gp_status fail(gp_ctx* ctx, const GpError& e) {
  if (ctx) ctx->err = e.msg;
  return e.st;
}

template <class F>
gp_status guarded(gp_ctx* ctx, F&& body) {
  try {
    if (ctx) GP_CUDA(cudaSetDevice(ctx->device));
    body();
    if (ctx) ctx->err.clear();
    return GP_OK;
  } catch (const GpError& e) {
    return fail(ctx, e);
  } catch (const std::bad_alloc&) {
    return fail(ctx, GpError{GP_ERR_NOMEM, "host allocation failed"});
  } catch (const std::exception& e) {
    return fail(ctx, GpError{GP_ERR_STATE, e.what()});
  }
}

template <class T>
T* upload(gp_ctx* ctx, std::vector<DevBuf>& owner, const std::vector<T>& v) {
  T* p = dalloc<T>(ctx, owner, std::max<size_t>(v.size(), 1));
  if (!v.empty()) h2d(ctx, p, v.data(), v.size());
  return p;
}

void check_hyper(const gp_pointset* ps, const gp_hyper& h, const gp_hyper& h0, const gp_core* core) {
  GP_REQUIRE(h.d == ps->d, "theta.d differs from the point set dimension");
  GP_REQUIRE(h.n1 >= 0 && h.n1 <= GP_MAX_N1 && h.n2 >= 0, "theta.n1 must be in 0..32 and n2 >= 0");
  GP_REQUIRE(h.bump_dims >= 0 && h.bump_dims <= h.d, "theta.bump_dims must be in 0..d");
  GP_REQUIRE(h.n1 == h0.n1 && h.n2 == h0.n2 && h.bump_dims == h0.bump_dims, "all proposals must share n1, n2, bump_dims");
  GP_REQUIRE(h.r0, "theta.r0 is required");
  const int kind = core ? core->kind : GP_CORE_WENDLAND;
  GP_REQUIRE(kind == GP_CORE_WENDLAND || kind == GP_CORE_PACIOREK, "unknown core kind");
  int64_t nb = (int64_t)h.n1 * h.n2;
  GP_REQUIRE(nb == 0 || (h.h && h.a && h.b && h.r), "bump arrays are required when n1*n2 > 0");
  if (kind == GP_CORE_WENDLAND) {
    GP_REQUIRE(ps->support == 0, "a point set assembled for the support of C_sparse needs the non-compact core");
    GP_REQUIRE(h.core_radius, "theta.core_radius is required");
    for (int k = 0; k < h.d; k++) {
      GP_REQUIRE(h.core_radius[k] == ps->rho[k], "theta.core_radius must equal the radii of gp_assemble");
      GP_REQUIRE(h.r0[k] > 0.0, "theta.r0 must be positive");
    }
  } else {
    GP_REQUIRE(ps->support == 1, "the non-compact core needs a point set from gp_assemble_sparse_support");
    GP_REQUIRE(h.n1 == ps->sup_n1 && h.n2 == ps->sup_n2 && h.bump_dims == ps->sup_bd,
               "theta's bump counts differ from the point set's support");
    for (int k = 0; k < h.d; k++) GP_REQUIRE(h.r0[k] == ps->rho[k], "theta.r0 must equal the point set's r0");
    for (int64_t q = 0; q < nb * h.bump_dims; q++) GP_REQUIRE(h.h[q] == ps->sup_h[q], "theta.h must equal the point set's");
    for (int64_t q = 0; q < nb; q++) GP_REQUIRE(h.r[q] == ps->sup_r[q], "theta.r must equal the point set's");
    GP_REQUIRE(core->phi_sigma && core->phi_Sigma, "core.phi_sigma and core.phi_Sigma are required");
    GP_REQUIRE(core->sigma0 > 0.0 && core->Sigma0 > 0.0 && std::isfinite(core->sigma0) && std::isfinite(core->Sigma0),
               "core.sigma0 and core.Sigma0 must be positive");
    for (int k = 0; k < h.d; k++)
      GP_REQUIRE(std::isfinite(core->phi_sigma[k]) && std::isfinite(core->phi_Sigma[k]), "non-finite core.phi");
  }
  GP_REQUIRE(std::isfinite(h.core_var) && std::isfinite(h.s0) && std::isfinite(h.noise_var), "non-finite theta");
}

void pack_thetas(gp_factor_t* f, const gp_hyper* th, const gp_core* cores) {
  const gp_hyper& h0 = th[0];
  ThetaDims td{h0.d, h0.n1, h0.n2, h0.bump_dims};
  int64_t st = theta_stride_of(td);
  std::vector<double> buf((size_t)st * f->B, 0.0);
  const int kind0 = cores ? cores[0].kind : GP_CORE_WENDLAND;
  for (int b = 0; b < f->B; b++) {
    const gp_hyper& h = th[b];
    const gp_core* c = cores ? &cores[b] : nullptr;
    check_hyper(f->ps, h, h0, c);
    GP_REQUIRE((c ? c->kind : GP_CORE_WENDLAND) == kind0, "all settings of a factor must share the core kind");
    double* p = buf.data() + (size_t)st * b;
    p[TH_CORE_VAR] = h.core_var;
    p[TH_S0] = h.s0;
    p[TH_NOISE] = h.noise_var;
    for (int k = 0; k < 3; k++) {
      p[TH_CRAD + k] = k < h.d ? (kind0 == GP_CORE_PACIOREK ? h.r0[k] : h.core_radius[k]) : 1.0;
      p[TH_R0 + k] = k < h.d ? h.r0[k] : 1.0;
    }
    p[TH_KIND] = kind0;
    if (kind0 == GP_CORE_PACIOREK) {
      p[TH_SIG0] = c->sigma0;
      p[TH_SIGMA0] = c->Sigma0;
      for (int k = 0; k < 3; k++) {
        p[TH_PHIS + k] = k < h.d ? c->phi_sigma[k] : 0.0;
        p[TH_PHIS2 + k] = k < h.d ? c->phi_Sigma[k] : 0.0;
      }
    }
    int64_t nb = (int64_t)h.n1 * h.n2;
    double* q = p + TH_BUMPS;
    for (int64_t ij = 0; ij < nb; ij++) {
      for (int k = 0; k < h.bump_dims; k++) *q++ = h.h[ij * h.bump_dims + k];
      *q++ = h.a[ij];
      *q++ = h.b[ij];
      *q++ = h.r[ij];
    }
  }
  f->theta_stride = st;
  f->n1max = h0.n1;
  GP_REQUIRE(f->core_kind == kind0, "the settings' core kind differs from the factor's");
  h2d(f->ctx, f->theta_dev, buf.data(), buf.size());
  GP_CUDA(cudaStreamSynchronize(f->ctx->stream));   // buf leaves scope
  f->thetas_host.assign(th, th + f->B);
}

}  // namespace

// ------------------------------------------------------------------------------------------ context
extern "C" gp_status gp_create(gp_ctx** out, int device, void* cuda_stream, size_t mem_budget_bytes) {
  if (!out) return GP_ERR_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return GP_ERR_ARG;
  }
  gp_ctx* ctx = new gp_ctx();
  ctx->device = device;
  ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  ctx->budget = mem_budget_bytes;
  gp_status st = guarded(ctx, [&] {
    GP_CUDA(cudaSetDevice(device));
    GP_CUDA(cudaFree(nullptr));
    GP_CUDA(cudaDeviceGetAttribute(&ctx->nsm, cudaDevAttrMultiProcessorCount, device));
    if (ctx->stream) {
      GP_CUDA(cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking));
      GP_CUDA(cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming));
      GP_CUDA(cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming));
      GP_CUDA(cudaStreamCreateWithFlags(&ctx->side2, cudaStreamNonBlocking));
      GP_CUDA(cudaEventCreateWithFlags(&ctx->ev_fork2, cudaEventDisableTiming));
      GP_CUDA(cudaEventCreateWithFlags(&ctx->ev_join2, cudaEventDisableTiming));
    }
  });
  if (st != GP_OK) {
    delete ctx;
    return st;
  }
  *out = ctx;
  return GP_OK;
}

namespace {
// A handle keeps its context alive: gp_destroy before the last *_free only marks the context.
void ctx_release(gp_ctx* ctx) {
  if (--ctx->live == 0 && ctx->destroyed) delete ctx;
}
}  // namespace

extern "C" void gp_destroy(gp_ctx* ctx) {
  if (!ctx) return;
  ctx->destroyed = true;
  if (ctx->live == 0) delete ctx;
}

extern "C" const char* gp_last_error(const gp_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

extern "C" int64_t gp_launch_count(const gp_ctx* ctx) { return ctx ? ctx->launches : 0; }

extern "C" gp_status gp_set_option(gp_ctx* ctx, int option, int64_t value) {
  if (!ctx) return GP_ERR_ARG;
  switch (option) {
    case GP_OPT_DIAG_FP32:
      if (value != 0 && value != 1) return fail(ctx, GpError{GP_ERR_ARG, "GP_OPT_DIAG_FP32 takes 0 or 1"});
      ctx->opt_diag_fp32 = (int)value;
      return GP_OK;
    case GP_OPT_WAIT_POLLS:
      if (value < 1 || value > 0xffffffffLL) return fail(ctx, GpError{GP_ERR_ARG, "GP_OPT_WAIT_POLLS takes 1..2^32-1"});
      ctx->opt_wait.polls = (uint32_t)value;
      return GP_OK;
    case GP_OPT_WAIT_NS:
      if (value < 0) return fail(ctx, GpError{GP_ERR_ARG, "GP_OPT_WAIT_NS takes a value >= 0"});
      ctx->opt_wait.ns = (uint64_t)value;
      return GP_OK;
    case GP_OPT_REFINE_EXP:
      if (value < 6 || value > 15) return fail(ctx, GpError{GP_ERR_ARG, "GP_OPT_REFINE_EXP takes 6..15"});
      ctx->opt_refine_exp = (int)value;
      return GP_OK;
    case GP_OPT_SPLIT_F16:
      if (value != 0 && value != 1) return fail(ctx, GpError{GP_ERR_ARG, "GP_OPT_SPLIT_F16 takes 0 or 1"});
      ctx->opt_split_f16 = (int)value;
      return GP_OK;
    default:
      return fail(ctx, GpError{GP_ERR_ARG, "unknown option " + std::to_string(option)});
  }
}

extern "C" gp_status gp_get_option(const gp_ctx* ctx, int option, int64_t* value) {
  if (!ctx || !value) return GP_ERR_ARG;
  switch (option) {
    case GP_OPT_DIAG_FP32: *value = ctx->opt_diag_fp32; return GP_OK;
    case GP_OPT_WAIT_POLLS: *value = (int64_t)ctx->opt_wait.polls; return GP_OK;
    case GP_OPT_WAIT_NS: *value = (int64_t)ctx->opt_wait.ns; return GP_OK;
    case GP_OPT_REFINE_EXP: *value = ctx->opt_refine_exp; return GP_OK;
    case GP_OPT_SPLIT_F16: *value = ctx->opt_split_f16; return GP_OK;
    default: return GP_ERR_ARG;
  }
}

namespace {
void prof_collect(gp_ctx* ctx) {
  cudaStreamSynchronize(ctx->stream);
  for (int k = 0; k < KC_COUNT; k++) {
    for (size_t e = 0; e < ctx->prof_ev[k].size(); e++) {
      const auto& ev = ctx->prof_ev[k][e];
      const int lv = e < ctx->prof_lv[k].size() ? ctx->prof_lv[k][e] : -1;
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, ev.first, ev.second) == cudaSuccess) {
        ctx->prof_ms[k] += ms;
        if (lv >= 0 && lv < GP_PROF_LEVELS) ctx->prof_ms_lv[k][lv] += ms;
      }
      if (lv >= 0 && lv < GP_PROF_LEVELS) ctx->prof_n_lv[k][lv]++;
      cudaEventDestroy(ev.first);
      cudaEventDestroy(ev.second);
    }
    ctx->prof_ev[k].clear();
    ctx->prof_lv[k].clear();
  }
}
}  // namespace

extern "C" gp_status gp_profile(gp_ctx* ctx, int enable) {
  if (!ctx) return GP_ERR_ARG;
  return guarded(ctx, [&] {
    prof_collect(ctx);
    for (int k = 0; k < KC_COUNT; k++) {
      ctx->prof_ms[k] = 0.0;
      ctx->prof_n[k] = 0;
      ctx->prof_flops[k] = 0.0;
      for (int l = 0; l < GP_PROF_LEVELS; l++) {
        ctx->prof_ms_lv[k][l] = 0.0;
        ctx->prof_n_lv[k][l] = 0;
      }
    }
    ctx->prof = enable != 0;
  });
}

extern "C" gp_status gp_profile_read(gp_ctx* ctx, int kclass, double* total_ms, int64_t* launches, double* flops) {
  if (!ctx || kclass < 0 || kclass >= KC_COUNT) return GP_ERR_ARG;
  return guarded(ctx, [&] {
    prof_collect(ctx);
    if (total_ms) *total_ms = ctx->prof_ms[kclass];
    if (launches) *launches = ctx->prof_n[kclass];
    if (flops) *flops = ctx->prof_flops[kclass];
  });
}

extern "C" gp_status gp_profile_read_level(gp_ctx* ctx, int kclass, int level, double* total_ms,
                                           int64_t* launches) {
  if (!ctx || kclass < 0 || kclass >= KC_COUNT || level < 0 || level >= GP_PROF_LEVELS) return GP_ERR_ARG;
  return guarded(ctx, [&] {
    prof_collect(ctx);
    if (total_ms) *total_ms = ctx->prof_ms_lv[kclass][level];
    if (launches) *launches = ctx->prof_n_lv[kclass][level];
  });
}

// ------------------------------------------------------------------------------------------ point sets
namespace {
gp_status assemble_common(gp_ctx* ctx, const double* d_X, int64_t n, int d, const double* core_radius,
                          const gp_hyper* support, gp_pointset** out);
}  // namespace

extern "C" gp_status gp_assemble(gp_ctx* ctx, const double* d_X, int64_t n, int d, const double* core_radius,
                                 gp_pointset** out) {
  return assemble_common(ctx, d_X, n, d, core_radius, nullptr, out);
}

extern "C" gp_status gp_assemble_sparse_support(gp_ctx* ctx, const double* d_X, int64_t n, int d,
                                                const gp_hyper* theta, gp_pointset** out) {
  if (!ctx) return GP_ERR_ARG;
  if (!theta || !theta->r0) return fail(ctx, GpError{GP_ERR_ARG, "theta and theta.r0 are required"});
  return assemble_common(ctx, d_X, n, d, theta->r0, theta, out);
}

namespace {
gp_status assemble_common(gp_ctx* ctx, const double* d_X, int64_t n, int d, const double* core_radius,
                          const gp_hyper* support, gp_pointset** out) {
  if (!ctx) return GP_ERR_ARG;
  if (!out) return fail(ctx, GpError{GP_ERR_ARG, "ps is null"});
  *out = nullptr;
  gp_pointset* ps = new gp_pointset();
  gp_status st = guarded(ctx, [&] {
    GP_REQUIRE(d_X && core_radius, "d_X and core_radius are required");
    GP_REQUIRE(n >= 1 && n < ((int64_t)1 << 31) - 1, "n must be in 1..2^31-2");
    GP_REQUIRE(d >= 1 && d <= GP_MAX_D, "d must be 1, 2 or 3");
    for (int k = 0; k < d; k++) GP_REQUIRE(core_radius[k] > 0.0 && std::isfinite(core_radius[k]), "core_radius must be positive");
    ps->ctx = ctx;
    ps->n = n;
    ps->d = d;
    for (int k = 0; k < d; k++) ps->rho[k] = core_radius[k];
    if (support) {   // the support of C_sparse: r0 (the grid unit) and the bumps' centres and radii
      const gp_hyper& h = *support;
      GP_REQUIRE(h.d == d, "theta.d differs from d");
      GP_REQUIRE(h.n1 >= 0 && h.n1 <= GP_MAX_N1 && h.n2 >= 0 && h.bump_dims >= 0 && h.bump_dims <= d,
                 "theta.n1 must be in 0..32, n2 >= 0 and bump_dims in 0..d");
      const int64_t nb = (int64_t)h.n1 * h.n2;
      GP_REQUIRE(nb == 0 || (h.h && h.r), "bump centres and radii are required");
      ps->support = 1;
      ps->sup_n1 = h.n1;
      ps->sup_n2 = h.n2;
      ps->sup_bd = h.bump_dims;
      ps->sup_h.assign(h.h, h.h + nb * h.bump_dims);
      ps->sup_r.assign(h.r, h.r + nb);
    }
    assemble_pointset(ctx, ps, d_X);       // A1, A2, A5 on the device
    // A6 on the host from the device pattern and order
    std::vector<int64_t> rp(n + 1);
    std::vector<int32_t> col(ps->nnz), perm(n);
    d2h(ctx, rp.data(), ps->rowptr, n + 1);
    d2h(ctx, col.data(), ps->col, ps->nnz);
    d2h(ctx, perm.data(), ps->perm, n);
    GP_CUDA(cudaStreamSynchronize(ctx->stream));
    build_symbolic(n, rp.data(), col.data(), perm.data(), ps->sp);
    SymPlan& sp = ps->sp;
    h2d(ctx, ps->perm, sp.perm.data(), n);
    DevPlan& dp = ps->dp;
    dp.w = upload(ctx, ps->bufs, sp.sn_w);
    dp.r = upload(ctx, ps->bufs, sp.sn_r);
    dp.loff = upload(ctx, ps->bufs, sp.sn_loff);
    dp.uoff = upload(ctx, ps->bufs, sp.sn_uoff);
    dp.frow_off = upload(ctx, ps->bufs, sp.sn_frow);
    dp.frows = upload(ctx, ps->bufs, sp.frows);
    dp.ch_ptr = upload(ctx, ps->bufs, sp.ch_ptr);
    dp.ch_idx = upload(ctx, ps->bufs, sp.ch_idx);
    dp.relidx_off = upload(ctx, ps->bufs, sp.relidx_off);
    dp.relidx = upload(ctx, ps->bufs, sp.relidx);
    dp.sn_first = upload(ctx, ps->bufs, sp.sn_first);
    dp.sn_of_col = upload(ctx, ps->bufs, sp.sn_of_col);
    dp.ea_tab = upload(ctx, ps->bufs, sp.ea_tab);
    dp.ea32_tab = upload(ctx, ps->bufs, sp.ea32_tab);
    dp.zero_tab = upload(ctx, ps->bufs, sp.zero_tab);
    dp.small_list = upload(ctx, ps->bufs, sp.small_list);
    dp.large_fronts = upload(ctx, ps->bufs, sp.large_fronts);
    dp.step_pre = upload(ctx, ps->bufs, sp.step_pre);
    dp.pair_pre = upload(ctx, ps->bufs, sp.pair_pre);
    dp.lev_sn = upload(ctx, ps->bufs, sp.lev_sn);
    dp.sn_parent = upload(ctx, ps->bufs, sp.sn_parent);
    dp.ldw = upload(ctx, ps->bufs, sp.sn_ldw);
    dp.loff32 = upload(ctx, ps->bufs, sp.sn_loff32);
    dp.lo_off = upload(ctx, ps->bufs, sp.sn_lo_off);
    dp.doff = upload(ctx, ps->bufs, sp.sn_doff);
    dp.large_kb = upload(ctx, ps->bufs, sp.large_kb);
    dp.sn_fl = upload(ctx, ps->bufs, sp.sn_fl);
    dp.flow_fwd = upload(ctx, ps->bufs, sp.flow_fwd);
    dp.flow_bwd = upload(ctx, ps->bufs, sp.flow_bwd);
    upload_schedule(ctx, ps);
    compute_dest_map(ctx, ps);             // pinv and the CSR -> panel scatter map
    GP_CUDA(cudaStreamSynchronize(ctx->stream));
  });
  if (st != GP_OK) {
    dev_free_all(ctx, ps->sched_bufs);
    dev_free_all(ctx, ps->bufs);
    delete ps;
    return st;
  }
  ctx->live++;
  *out = ps;
  return GP_OK;
}
}  // namespace

extern "C" void gp_pointset_free(gp_pointset* ps) {
  if (!ps) return;
  gp_ctx* ctx = ps->ctx;
  if (ctx) {
    cudaSetDevice(ctx->device);
    dev_free_all(ctx, ps->sched_bufs);
    dev_free_all(ctx, ps->bufs);
  }
  delete ps;
  if (ctx) ctx_release(ctx);
}

extern "C" gp_status gp_pointset_info(const gp_pointset* ps, gp_pointset_info_t* info) {
  if (!ps || !info) return GP_ERR_ARG;
  const SymPlan& sp = ps->sp;
  info->n = ps->n;
  info->d = ps->d;
  info->nnz = ps->nnz;
  info->ncells = ps->ncells;
  info->nnzL = sp.nnzL;
  info->nsuper = sp.ns;
  info->panel_entries = sp.panel_entries;
  info->update_entries = sp.update_entries;
  info->nlevels = sp.nlevels;
  info->max_front = sp.max_front;
  info->flops = sp.flops;
  return GP_OK;
}

extern "C" gp_status gp_pointset_export(const gp_pointset* ps, int what, void* dst, size_t bytes) {
  if (!ps || !dst) return GP_ERR_ARG;
  gp_ctx* ctx = ps->ctx;
  const SymPlan& sp = ps->sp;
  auto host = [&](const void* src, size_t b) -> gp_status {
    if (b != bytes) return fail(ctx, GpError{GP_ERR_ARG, "export size mismatch: expected " + std::to_string(b)});
    if (b) memcpy(dst, src, b);
    return GP_OK;
  };
  auto dev = [&](const void* src, size_t b) -> gp_status {
    if (b != bytes) return fail(ctx, GpError{GP_ERR_ARG, "export size mismatch: expected " + std::to_string(b)});
    return guarded(ctx, [&] {
      GP_CUDA(cudaMemcpyAsync(dst, src, b, cudaMemcpyDeviceToHost, ctx->stream));
      GP_CUDA(cudaStreamSynchronize(ctx->stream));
    });
  };
  const size_t n = (size_t)ps->n;
  switch (what) {
    case 0: return host(sp.perm.data(), n * 4);
    case 1: return host(sp.parent.data(), n * 4);
    case 2: return host(sp.eta.data(), n * 4);
    case 3: return dev(ps->rowptr, (n + 1) * 8);
    case 4: return dev(ps->col, (size_t)ps->nnz * 4);
    case 5: return host(sp.sn_first.data(), sp.sn_first.size() * 4);
    case 6: return host(sp.sn_rowptr.data(), sp.sn_rowptr.size() * 8);
    case 7: return host(sp.sn_rows.data(), sp.sn_rows.size() * 4);
    case 8: return host(sp.sn_parent.data(), sp.sn_parent.size() * 4);
    case 9: return host(sp.sn_level.data(), sp.sn_level.size() * 4);
    case 10: return dev(ps->cell_perm, n * 4);
    default: return fail(ctx, GpError{GP_ERR_ARG, "unknown export"});
  }
}

// ------------------------------------------------------------------------------------------ host symbolic
struct gp_symbolic {
  int64_t n = 0, nnz = 0;
  SymPlan sp;
};

extern "C" gp_status gp_symbolic_host(int64_t n, const int64_t* rowptr, const int32_t* col, const int32_t* nd_perm,
                                      gp_symbolic** out) {
  if (!out) return GP_ERR_ARG;
  *out = nullptr;
  if (!rowptr || !col || !nd_perm || n < 1 || n >= ((int64_t)1 << 31) - 1 || rowptr[0] != 0) return GP_ERR_ARG;
  for (int64_t i = 0; i < n; i++) {   // the pattern: ascending in-range columns, the diagonal present
    if (rowptr[i + 1] < rowptr[i]) return GP_ERR_ARG;
    bool diag = false;
    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; e++) {
      if (col[e] < 0 || col[e] >= n || (e > rowptr[i] && col[e] <= col[e - 1])) return GP_ERR_ARG;
      diag = diag || col[e] == i;
    }
    if (!diag) return GP_ERR_ARG;
  }
  try {
    std::vector<char> seen((size_t)n, 0);
    for (int64_t k = 0; k < n; k++) {
      const int32_t v = nd_perm[k];
      if (v < 0 || v >= n || seen[v]) return GP_ERR_ARG;
      seen[v] = 1;
    }
    std::unique_ptr<gp_symbolic> s(new gp_symbolic);
    s->n = n;
    s->nnz = rowptr[n];
    build_symbolic(n, rowptr, col, nd_perm, s->sp);
    *out = s.release();
    return GP_OK;
  } catch (const GpError& e) {
    return e.st;
  } catch (const std::bad_alloc&) {
    return GP_ERR_NOMEM;
  } catch (const std::exception&) {
    return GP_ERR_STATE;
  }
}

extern "C" gp_status gp_symbolic_info(const gp_symbolic* sym, gp_pointset_info_t* info) {
  if (!sym || !info) return GP_ERR_ARG;
  const SymPlan& sp = sym->sp;
  *info = gp_pointset_info_t{};
  info->n = sym->n;
  info->nnz = sym->nnz;
  info->nnzL = sp.nnzL;
  info->nsuper = sp.ns;
  info->panel_entries = sp.panel_entries;
  info->update_entries = sp.update_entries;
  info->nlevels = sp.nlevels;
  info->max_front = sp.max_front;
  info->flops = sp.flops;
  return GP_OK;
}

extern "C" gp_status gp_symbolic_export(const gp_symbolic* sym, int what, void* dst, size_t bytes) {
  if (!sym || !dst) return GP_ERR_ARG;
  const SymPlan& sp = sym->sp;
  auto host = [&](const void* src, size_t b) -> gp_status {
    if (b != bytes) return GP_ERR_ARG;
    if (b) memcpy(dst, src, b);
    return GP_OK;
  };
  const size_t n = (size_t)sym->n;
  switch (what) {
    case 0: return host(sp.perm.data(), n * 4);
    case 1: return host(sp.parent.data(), n * 4);
    case 2: return host(sp.eta.data(), n * 4);
    case 5: return host(sp.sn_first.data(), sp.sn_first.size() * 4);
    case 6: return host(sp.sn_rowptr.data(), sp.sn_rowptr.size() * 8);
    case 7: return host(sp.sn_rows.data(), sp.sn_rows.size() * 4);
    case 8: return host(sp.sn_parent.data(), sp.sn_parent.size() * 4);
    case 9: return host(sp.sn_level.data(), sp.sn_level.size() * 4);
    default: return GP_ERR_ARG;
  }
}

extern "C" void gp_symbolic_free(gp_symbolic* sym) { delete sym; }

// The mixed-path update schedule on the device (replaced when it is re-planned).
void upload_schedule(gp_ctx* ctx, gp_pointset* ps) {
  dev_free_all(ctx, ps->sched_bufs);
  ps->dp.upd_fronts = upload(ctx, ps->sched_bufs, ps->sp.upd_fronts);
  ps->dp.upd_pre = upload(ctx, ps->sched_bufs, ps->sp.upd_pre);
  GP_CUDA(cudaStreamSynchronize(ctx->stream));
}

// ------------------------------------------------------------------------------------------ factors
extern "C" gp_status gp_factor(gp_ctx* ctx, gp_pointset* ps, const gp_hyper* thetas, int B, gp_precision prec,
                               gp_factor_t** out) {
  return gp_factor_core(ctx, ps, thetas, nullptr, B, prec, out);
}

extern "C" gp_status gp_factor_core(gp_ctx* ctx, gp_pointset* ps, const gp_hyper* thetas, const gp_core* cores,
                                    int B, gp_precision prec, gp_factor_t** out) {
  if (!ctx) return GP_ERR_ARG;
  if (!out) return fail(ctx, GpError{GP_ERR_ARG, "f is null"});
  *out = nullptr;
  gp_factor_t* f = new gp_factor_t();
  gp_status st = guarded(ctx, [&] {
    GP_REQUIRE(ps && ps->ctx && ps->ctx->device == ctx->device, "point set missing or on another device");
    GP_REQUIRE(thetas && B >= 1, "B >= 1 settings are required");
    GP_REQUIRE(prec == GP_FP64 || prec == GP_MIXED, "unknown precision");
    const SymPlan& sp = ps->sp;
    f->ctx = ctx;
    f->ps = ps;
    f->B = B;
    f->prec = prec;
    f->diag_fp32 = prec == GP_MIXED && ctx->opt_diag_fp32 != 0;
    f->op_f16 = prec == GP_MIXED && ctx->opt_split_f16 != 0;
    f->wait_lim = ctx->opt_wait;
    f->refine_tol = std::pow(10.0, -(double)ctx->opt_refine_exp);
    f->core_kind = cores ? cores[0].kind : GP_CORE_WENDLAND;
    ThetaDims td{thetas[0].d, thetas[0].n1, thetas[0].n2, thetas[0].bump_dims};
    GP_REQUIRE(td.d == ps->d, "theta.d differs from the point set dimension");
    GP_REQUIRE(td.n1 >= 0 && td.n1 <= GP_MAX_N1, "n1 must be in 0..32");
    f->theta_dev = dalloc<double>(ctx, f->bufs, (size_t)theta_stride_of(td) * B);
    f->F = dalloc<double>(ctx, f->bufs, (size_t)B * ps->n * td.n1 + 1);
    if (f->core_kind == GP_CORE_PACIOREK) f->Cpt = dalloc<double>(ctx, f->bufs, (size_t)B * ps->n * 2);
    if (prec == GP_FP64) {
      f->panels = dalloc<double>(ctx, f->bufs, (size_t)B * sp.panel_entries);
      f->upd = dalloc<double>(ctx, f->bufs, (size_t)B * sp.update_entries);
    } else {
      if (!ps->dest32) {   // the point set's own context owns (and stream-orders) its per-precision map
        compute_dest_map_mixed(ps->ctx, ps);
        GP_CUDA(cudaStreamSynchronize(ps->ctx->stream));
      }
      f->panels32 = dalloc<float>(ctx, f->bufs, (size_t)B * sp.panel32_entries);
      f->diag = dalloc<double>(ctx, f->bufs, (size_t)B * sp.diag_entries);
      f->upd32 = dalloc<float>(ctx, f->bufs, (size_t)B * sp.update_entries);
      f->delta = dalloc<double>(ctx, f->bufs, (size_t)B * ps->n * 2);
      f->ll_buf = dalloc<double>(ctx, f->bufs, (size_t)2 * B);
      f->refine_it = dalloc<int32_t>(ctx, f->bufs, 1);
      f->refine_runs = dalloc<unsigned long long>(ctx, f->bufs, 1);
      GP_CUDA(cudaMemsetAsync(f->refine_runs, 0, sizeof(unsigned long long), ctx->stream));
      f->dinv32 = dalloc<float>(ctx, f->bufs, (size_t)B * sp.diag_entries);
      f->op_lo = dalloc<float>(ctx, f->bufs, (size_t)B * sp.lo_entries);
      GP_CUDA(cudaMemsetAsync(f->op_lo, 0, (size_t)B * sp.lo_entries * sizeof(float), ctx->stream));
      f->op_dmax = dalloc<unsigned long long>(ctx, f->bufs, B);
      build_update_maps(ctx, f);
    }
    f->val = dalloc<double>(ctx, f->bufs, (size_t)B * ps->nnz);
    f->notpd = dalloc<int32_t>(ctx, f->bufs, B);
    f->alpha = dalloc<double>(ctx, f->bufs, (size_t)B * ps->n);
    if (prec == GP_FP64) f->dinv = dalloc<double>(ctx, f->bufs, (size_t)B * sp.diag_entries);
    f->rhs = dalloc<double>(ctx, f->bufs, (size_t)B * ps->n);
    f->work_stride = 3 * ps->n + sp.vec_update_entries + 64;
    f->work = dalloc<double>(ctx, f->bufs, (size_t)B * f->work_stride);
    f->bwd_part = dalloc<double>(ctx, f->bufs, (size_t)B * bwd_part_entries(sp));
    f->tiles_err = dalloc<int32_t>(ctx, f->bufs, 1);
    GP_CUDA(cudaMemsetAsync(f->tiles_err, 0, sizeof(int32_t), ctx->stream));
    f->flow_sync = dalloc<int32_t>(ctx, f->bufs, flow_sync_entries(sp, B));
    f->red_stride = 2 * ((ps->n + 1023) / 1024) + 8;
    f->red = dalloc<double>(ctx, f->bufs, (size_t)B * f->red_stride + 4 * (size_t)B + 8);
    pack_thetas(f, thetas, cores);
    factor_run(ctx, f);
  });
  if (st != GP_OK) {
    dev_free_all(ctx, f->bufs);
    for (cudaGraphExec_t g : {f->gx_factor, f->gx_solve, f->gx_cor, f->gx_refine, f->gx_tail})
      if (g) cudaGraphExecDestroy(g);
    delete f;
    return st;
  }
  ctx->live++;
  ps->nfactors++;
  *out = f;
  return GP_OK;
}

namespace {
size_t alloc_bytes(size_t b) { return ((b == 0 ? 16 : b) + 255) & ~size_t(255); }
}  // namespace

// Device bytes gp_factor allocates for (ps, prec, B): the same list of buffers, rounded as dev_alloc rounds.
size_t factor_bytes(const gp_pointset* ps, gp_precision prec, int B, const ThetaDims& td) {
  const SymPlan& sp = ps->sp;
  const size_t b = (size_t)B, n = (size_t)ps->n;
  size_t t = alloc_bytes((size_t)theta_stride_of(td) * b * 8) + alloc_bytes((b * n * td.n1 + 1) * 8);
  if (ps->support == 1) t += alloc_bytes(b * n * 2 * 8);   // the non-compact core's per-point sigma, Sigma
  if (prec == GP_FP64) {
    t += alloc_bytes(b * sp.panel_entries * 8) + alloc_bytes(b * sp.update_entries * 8);
  } else {
    std::vector<char> seen(sp.sn_w.size(), 0);
    size_t nmaps = 0;
    for (int32_t s : sp.large_fronts)
      if (!seen[s]) {
        seen[s] = 1;
        nmaps++;
      }
    nmaps = std::max<size_t>(nmaps, 1);
    t += alloc_bytes(b * sp.panel32_entries * 4) + alloc_bytes(b * sp.diag_entries * 8) +
         alloc_bytes(b * sp.update_entries * 4) + alloc_bytes(b * n * 2 * 8) + alloc_bytes(4) +
         alloc_bytes(8) +
         alloc_bytes(b * sp.diag_entries * 4) + alloc_bytes(b * sp.lo_entries * 4) +
         alloc_bytes(b * 8) + alloc_bytes(2 * nmaps * 128) + alloc_bytes((sp.sn_w.size() + 1) * 4) +
         alloc_bytes(b * 2 * 8);
  }
  t += alloc_bytes(b * ps->nnz * 8) + alloc_bytes(b * 4) + alloc_bytes(b * n * 8);
  if (prec == GP_FP64) t += alloc_bytes(b * sp.diag_entries * 8);
  t += alloc_bytes(b * n * 8) + alloc_bytes(b * (3 * n + sp.vec_update_entries + 64) * 8) +
       alloc_bytes(b * (size_t)bwd_part_entries(sp) * 8) +
       alloc_bytes(4) + alloc_bytes((size_t)flow_sync_entries(sp, (int)b) * 4) +
       alloc_bytes((b * (2 * ((n + 1023) / 1024) + 8) + 4 * b + 8) * 8);
  return t;
}

extern "C" gp_status gp_factor_bytes(const gp_pointset* ps, const gp_hyper* theta, int B, gp_precision prec,
                                     size_t* bytes) {
  if (!ps || !theta || !bytes || B < 1 || (prec != GP_FP64 && prec != GP_MIXED)) return GP_ERR_ARG;
  if (theta->n1 < 0 || theta->n1 > GP_MAX_N1 || theta->d != ps->d) return GP_ERR_ARG;
  *bytes = factor_bytes(ps, prec, B, ThetaDims{theta->d, theta->n1, theta->n2, theta->bump_dims});
  return GP_OK;
}

extern "C" gp_status gp_pointset_prepare(gp_ctx* ctx, gp_pointset* ps, gp_precision prec) {
  if (!ctx) return GP_ERR_ARG;
  return guarded(ctx, [&] {
    GP_REQUIRE(ps && ps->ctx == ctx, "point set missing or from another context");
    GP_REQUIRE(prec == GP_FP64 || prec == GP_MIXED, "unknown precision");
    if (prec == GP_MIXED && !ps->dest32) compute_dest_map_mixed(ctx, ps);
    GP_CUDA(cudaStreamSynchronize(ctx->stream));
  });
}

extern "C" gp_status gp_pointset_set_blocking(gp_ctx* ctx, gp_pointset* ps, int group_blocks, int group_tile_n) {
  if (!ctx) return GP_ERR_ARG;
  return guarded(ctx, [&] {
    GP_REQUIRE(ps && ps->ctx == ctx, "point set missing or from another context");
    GP_REQUIRE(group_blocks >= 1 && group_blocks <= 64, "group_blocks must be in 1..64");
    GP_REQUIRE(group_tile_n == 128 || group_tile_n == 256, "group_tile_n must be 128 or 256");
    if (ps->nfactors.load() != 0) throw GpError{GP_ERR_STATE, "set the blocking before creating factors"};
    plan_mixed_updates(ps->sp, group_blocks, group_tile_n);
    upload_schedule(ctx, ps);
  });
}

extern "C" gp_status gp_autotune(gp_ctx* ctx, gp_pointset* ps, const gp_hyper* thetas, int B, int reps,
                                 gp_tune_candidate* tried, int* ntried) {
  if (!ctx) return GP_ERR_ARG;
  static const int cand[][2] = {{4, 128}, {4, 256}, {8, 128}, {8, 256}, {16, 128}, {16, 256}, {32, 256}};
  const int nc = (int)(sizeof(cand) / sizeof(cand[0]));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  gp_status st = guarded(ctx, [&] {
    GP_REQUIRE(ps && ps->ctx == ctx, "point set missing or from another context");
    if (ps->nfactors.load() != 0) throw GpError{GP_ERR_STATE, "tune a point set before creating its factors"};
    GP_REQUIRE(thetas && B >= 1 && reps >= 1, "B >= 1 settings and reps >= 1 are required");
    GP_CUDA(cudaEventCreate(&e0));
    GP_CUDA(cudaEventCreate(&e1));
    int best = -1;
    float best_ms = 0.f;
    for (int c = 0; c < nc; c++) {
      plan_mixed_updates(ps->sp, cand[c][0], cand[c][1]);
      upload_schedule(ctx, ps);
      gp_factor_t* f = nullptr;
      gp_status fs = gp_factor(ctx, ps, thetas, B, GP_MIXED, &f);   // allocates and factors once (graph capture)
      if (fs != GP_OK) throw GpError{fs, ctx->err};
      GP_CUDA(cudaEventRecord(e0, ctx->stream));
      for (int r = 0; r < reps && fs == GP_OK; r++) fs = gp_factor_update(ctx, f, thetas);
      GP_CUDA(cudaEventRecord(e1, ctx->stream));
      GP_CUDA(cudaEventSynchronize(e1));
      gp_factor_free(f);
      if (fs != GP_OK) throw GpError{fs, ctx->err};
      float ms = 0.f;
      GP_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      ms /= (float)reps;
      if (tried) tried[c] = gp_tune_candidate{cand[c][0], cand[c][1], (double)ms};
      if (best < 0 || ms < best_ms) {
        best = c;
        best_ms = ms;
      }
    }
    plan_mixed_updates(ps->sp, cand[best][0], cand[best][1]);
    upload_schedule(ctx, ps);
    if (ntried) *ntried = nc;
  });
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st != GP_OK && ps && ps->ctx == ctx && ps->nfactors.load() == 0) {   // leave the default blocking behind
    const std::string msg = ctx->err;
    guarded(ctx, [&] {
      plan_mixed_updates(ps->sp, GP_GROUP, GP_TN_GROUP);
      upload_schedule(ctx, ps);
    });
    ctx->err = msg;
  }
  return st;
}

extern "C" gp_status gp_factor_update(gp_ctx* ctx, gp_factor_t* f, const gp_hyper* thetas) {
  return gp_factor_update_core(ctx, f, thetas, nullptr);
}

extern "C" gp_status gp_factor_update_core(gp_ctx* ctx, gp_factor_t* f, const gp_hyper* thetas, const gp_core* cores) {
  if (!ctx) return GP_ERR_ARG;
  return guarded(ctx, [&] {
    GP_REQUIRE(f && f->ctx == ctx, "factor missing or from another context");
    GP_REQUIRE(thetas, "thetas required");
    GP_REQUIRE(thetas[0].n1 == f->n1max, "n1 must match the factor");
    pack_thetas(f, thetas, cores);
    f->have_alpha = false;
    factor_run(ctx, f);
  });
}

extern "C" void gp_factor_free(gp_factor_t* f) {
  if (!f) return;
  if (f->ps) f->ps->nfactors--;
  gp_ctx* ctx = f->ctx;
  if (ctx) {
    cudaSetDevice(ctx->device);
    dev_free_all(ctx, f->bufs);
  }
  for (cudaGraphExec_t g : {f->gx_factor, f->gx_solve, f->gx_cor, f->gx_refine, f->gx_tail})
    if (g) cudaGraphExecDestroy(g);
  delete f;
  if (ctx) ctx_release(ctx);
}

extern "C" gp_status gp_factor_info(const gp_factor_t* f, gp_factor_info_t* info, int32_t* not_pd_column) {
  if (!f || !info) return GP_ERR_ARG;
  gp_ctx* ctx = f->ctx;
  std::vector<int32_t> flags(f->B);
  int32_t terr = 0;
  unsigned long long runs = 0;
  gp_status st = guarded(ctx, [&] {
    d2h(ctx, flags.data(), f->notpd, f->B);
    if (f->tiles_err) d2h(ctx, &terr, f->tiles_err, 1);
    if (f->refine_runs) d2h(ctx, &runs, f->refine_runs, 1);
    GP_CUDA(cudaStreamSynchronize(ctx->stream));
  });
  if (st != GP_OK) return st;
  if (runs > f->refine_runs_seen) {   // the refinement loop's passes, counted once they are known
    ctx->launches += (int64_t)(runs - f->refine_runs_seen) * f->n_refine_body;
    const_cast<gp_factor_t*>(f)->refine_runs_seen = runs;
  }
  info->timed_out = terr != 0 ? 1 : 0;
  info->B = f->B;
  info->precision = f->prec;
  int64_t bytes = 0;
  for (auto& b : f->bufs) bytes += (int64_t)b.bytes;
  info->bytes = bytes;
  info->not_pd_count = 0;
  info->diag_fp32 = f->diag_fp32 ? 1 : 0;
  info->split_f16 = f->op_f16 ? 1 : 0;
  for (int b = 0; b < f->B; b++) {   // flags hold the smallest failing permuted column, INT_MAX if none
    bool bad = flags[b] != 0x7fffffff;
    if (bad) info->not_pd_count++;
    if (not_pd_column) not_pd_column[b] = bad ? flags[b] : -1;
  }
  if (terr != 0)
    return fail(ctx, GpError{GP_ERR_TIMEOUT, "a bounded wait of the tensor-core updates or of a solve ran out"});
  return GP_OK;
}

// ------------------------------------------------------------------------------------------ solves
extern "C" gp_status gp_loglik(gp_ctx* ctx, gp_factor_t* f, const double* d_resid, double* d_out, double* d_err_est) {
  if (!ctx) return GP_ERR_ARG;
  return guarded(ctx, [&] {
    GP_REQUIRE(f && f->ctx == ctx, "factor missing or from another context");
    GP_REQUIRE(d_resid && d_out, "d_resid and d_out are required");
    loglik_run(ctx, f, d_resid, d_out, d_err_est);
    f->have_alpha = true;
  });
}

extern "C" gp_status gp_loglik_iterative(gp_ctx* ctx, gp_factor_t* f, int b, const double* d_resid,
                                         const double* d_probes, const double* d_x0, const gp_iterative_opts* opts,
                                         gp_iterative_result* result) {
  if (!ctx) return GP_ERR_ARG;
  return guarded(ctx, [&] {
    GP_REQUIRE(f && f->ctx == ctx, "factor missing or from another context");
    GP_REQUIRE(b >= 0 && b < f->B, "proposal index out of range");
    GP_REQUIRE(d_resid && d_probes && opts && result, "d_resid, d_probes, opts and result are required");
    GP_REQUIRE(opts->probes >= 1 && opts->probes <= 32, "probes must be in 1..32");
    GP_REQUIRE(opts->lanczos_steps >= 2 && opts->lanczos_steps <= 64, "lanczos_steps must be in 2..64");
    GP_REQUIRE(opts->tol > 0.0 && opts->max_iter >= 1, "tol > 0 and max_iter >= 1 are required");
    iterative_run(ctx, f, b, d_resid, d_probes, d_x0, *opts, result);
  });
}

extern "C" gp_status gp_predict_var(gp_ctx* ctx, gp_factor_t* f, int b, const double* d_Xtest, int64_t m,
                                    double* d_var) {
  if (!ctx) return GP_ERR_ARG;
  return guarded(ctx, [&] {
    GP_REQUIRE(f && f->ctx == ctx, "factor missing or from another context");
    GP_REQUIRE(b >= 0 && b < f->B, "proposal index out of range");
    GP_REQUIRE(m >= 0 && (m == 0 || (d_Xtest && d_var)), "d_Xtest and d_var are required");
    if (m > 0) variance_run(ctx, f, b, d_Xtest, m, d_var);
  });
}

extern "C" gp_status gp_predict(gp_ctx* ctx, gp_factor_t* f, int b, const double* d_Xtest, int64_t m,
                                const double* d_mu_test, double* d_mean) {
  if (!ctx) return GP_ERR_ARG;
  return guarded(ctx, [&] {
    GP_REQUIRE(f && f->ctx == ctx, "factor missing or from another context");
    GP_REQUIRE(b >= 0 && b < f->B, "proposal index out of range");
    GP_REQUIRE(m >= 0 && (m == 0 || (d_Xtest && d_mean)), "d_Xtest and d_mean are required");
    if (!f->have_alpha) throw GpError{GP_ERR_STATE, "gp_predict needs gp_loglik first (alpha = C_z^-1 r)"};
    if (m > 0) {
      refine_alpha_for_predict(ctx, f);   // GP_MIXED: alpha to 1e-12 (gp_loglik may have stopped earlier)
      predict_run(ctx, f, b, d_Xtest, m, d_mu_test, d_mean);
    }
  });
}
