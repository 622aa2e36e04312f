// isis_api.cu -- the C ABI of include/isis.h: argument checks, the model
// constants, the workspace cache, and dispatch to the per-model drivers.
#include <cmath>
#include <cstdio>
#include <mutex>
#include <vector>
#include <algorithm>
#include <cstring>
#include <string>

#include "isis_patch.cuh"
#include "isis_solver.cuh"

namespace isis {

isis_status run_poi(const SolveArgs& A);
isis_status run_sym(const SolveArgs& A);
isis_status run_fofr(const SolveArgs& A);

// ---------------------------------------------------------------------------
// Workspace cache: one hierarchy per (device, N, element size, coarsest size)
// ---------------------------------------------------------------------------

static std::vector<Workspace*> g_ws;

static void free_ws(Workspace* w) {
  for (void* p : w->owned) cudaFree(p);
  if (w->host) cudaFreeHost(w->host);
  delete w;
}

Workspace* get_workspace(int N, int esize, int ncoarse) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  for (Workspace* w : g_ws)
    if (w->N == N && w->esize == esize && w->device == dev && (N >> (w->nlev - 1)) == ncoarse) return w;
  Workspace* w = new Workspace();
  w->N = N;
  w->esize = esize;
  w->device = dev;
  int nlev = 1;
  while ((N >> (nlev - 1)) > ncoarse) ++nlev;
  w->nlev = nlev;
  auto alloc = [&](size_t bytes) -> void* {
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
    w->owned.push_back(p);
    return p;
  };
  bool ok = true;
  std::vector<void*>* arrays[6] = {&w->x, &w->x0, &w->sig, &w->eta, &w->B, &w->w};
  for (int l = 0; l < nlev && ok; ++l) {
    size_t nl = (size_t)(N >> l) * (N >> l) * (N >> l);
    for (auto* a : arrays) {
      // the finest level's buffers only serve the FP32 cycles
      void* p = (l == 0 && esize != 4) ? nullptr : alloc(nl * esize);
      if (!(l == 0 && esize != 4) && !p) ok = false;
      a->push_back(p);
    }
    void* pa = alloc(nl * esize);
    if (!pa) ok = false;
    w->aux.push_back(pa);
  }
  if (ok) {
    w->part = (double*)alloc(kNormBlocks * sizeof(double));
    w->part2 = (double*)alloc(kNormBlocks * sizeof(double));
    w->scal = (double*)alloc(8 * sizeof(double));
    w->iflags = (int*)alloc(8 * sizeof(int));
    ok = w->part && w->part2 && w->scal && w->iflags;
  }
  if (ok && cudaHostAlloc(&w->host, 256, cudaHostAllocMapped) != cudaSuccess) ok = false;
  if (ok && cudaHostGetDevicePointer((void**)&w->host_dev, w->host, 0) != cudaSuccess) ok = false;
  if (ok) {
    w->exptab_ff = (float2*)alloc(64 * sizeof(float2));
    float2 tab[64];
    ff_exp_table_fill(tab);
    ok = w->exptab_ff && cudaMemcpy(w->exptab_ff, tab, sizeof(tab), cudaMemcpyHostToDevice) == cudaSuccess;
  }
  if (!ok) {
    free_ws(w);
    cudaGetLastError();
    return nullptr;
  }
  g_ws.push_back(w);
  return w;
}

// a[0 .. n) = v, four values per thread (a 16-byte aligned workspace grid, n a multiple of 4).
__global__ void fill_f32(float* __restrict__ a, size_t n, float v) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (4 * t < n) reinterpret_cast<float4*>(a)[t] = make_float4(v, v, v, v);
}

isis_status sum_f32(Workspace* ws, const float* v, size_t n, cudaStream_t st) {
  ISIS_LAUNCH(KK_REDUCE, 4.0 * n, st, (sum_f32_partial<<<kNormBlocks, kNormThreads, 0, st>>>(v, n, ws->part2)));
  ISIS_LAUNCH(KK_REDUCE, 0.0, st, (reduce_final<<<1, kNormThreads, 0, st>>>(ws->part2, kNormBlocks, ws->scal + 1)));
  return ISIS_OK;
}

float* get_xalt(Workspace* w, int l) {
  if (l < 0 || l >= w->nlev || w->esize != 4) return nullptr;
  if ((int)w->xalt.size() < w->nlev) w->xalt.resize(w->nlev, nullptr);
  if (!w->xalt[l]) {
    const size_t nl = (size_t)(w->N >> l) * (w->N >> l) * (w->N >> l);
    void* p = nullptr;
    if (cudaMalloc(&p, nl * sizeof(float)) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    w->owned.push_back(p);
    w->xalt[l] = p;
  }
  return (float*)w->xalt[l];
}

bool ensure_fofr64(Workspace* w) {
  if (w->b64) return true;
  size_t n = (size_t)w->N * w->N * w->N;
  void *p = nullptr, *q = nullptr;
  if (cudaMalloc(&p, n * sizeof(double)) != cudaSuccess) { cudaGetLastError(); return false; }
  if (cudaMalloc(&q, n * sizeof(double)) != cudaSuccess) { cudaFree(p); cudaGetLastError(); return false; }
  w->owned.push_back(p);
  w->owned.push_back(q);
  w->b64 = (double*)p;
  w->s64 = (double*)q;
  return true;
}

// int64 accumulation buffer of the CIC deposit, cached per (device, N)
struct DepositBuf {
  int N, device;
  unsigned long long* acc;
};
static std::vector<DepositBuf> g_dep;

unsigned long long* get_deposit_buf(int N) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  for (auto& d : g_dep)
    if (d.N == N && d.device == dev) return d.acc;
  void* p = nullptr;
  if (cudaMalloc(&p, (size_t)N * N * N * sizeof(unsigned long long)) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  g_dep.push_back({N, dev, (unsigned long long*)p});
  return (unsigned long long*)p;
}

// three float N^3 arrays of the grid force, cached per (device, N)
static std::vector<DepositBuf> g_fgrid;

float* get_force_buf(int N) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  for (auto& d : g_fgrid)
    if (d.N == N && d.device == dev) return (float*)d.acc;
  void* p = nullptr;
  if (cudaMalloc(&p, (size_t)4 * N * N * N * sizeof(float)) != cudaSuccess) {  // float4 per cell
    cudaGetLastError();
    return nullptr;
  }
  g_fgrid.push_back({N, dev, (unsigned long long*)p});
  return (float*)p;
}

// ---------------------------------------------------------------------------
// Argument checks and model constants
// ---------------------------------------------------------------------------

static bool pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

static bool grid_ok(const isis_grid* g) {
  return g && pow2(g->N) && g->N >= 8 && g->N <= 1024 && g->box > 0 && std::isfinite(g->box) && g->H0 > 0 &&
         g->Omega_m > 0 && g->Omega_L >= 0;
}

static bool opts_resolve(const isis_mg_opts* o, isis_mg_opts* out, int N) {
  isis_mg_opts d = {2, 2, 4, 100, ISIS_F64, 2, ISIS_INIT_INPUT, 0};
  if (o) d = *o;
  if (d.nu1 < 0 || d.nu1 > 16 || d.nu2 < 0 || d.nu2 > 16) return false;
  if (d.n_coarsest != 2 && d.n_coarsest != 4) return false;
  if (d.n_coarsest * 2 > N) return false;
  if (d.max_cycles < 0 || d.max_cycles > 128) return false;
  if (d.prec != ISIS_F64 && d.prec != ISIS_F32 && d.prec != ISIS_F32_REFINE64) return false;
  if (d.inner_cycles < 1 || d.inner_cycles > 16) return false;
  if (d.init != ISIS_INIT_INPUT && d.init != ISIS_INIT_BACKGROUND && d.init != ISIS_INIT_LOCAL) return false;
  if (d.fmg != 0 && d.fmg != 1) return false;
  *out = d;
  return true;
}

// Constants of a scalar model (field form, fscale = 1) and the scale of its reference residual.
static bool model_coef(isis_model model, const isis_params* p, const isis_grid* grid, double a, Coef* c,
                       double* ref_scale) {
  const double H02 = grid->H0 * grid->H0;
  if (model == ISIS_SYMMETRON) {
    if (!(p->lambda0 > 0) || !(p->a_ssb > 0)) return false;
    // Sect. 4.1, Eq. (symmetron_dimensionles)
    c->A = a * a / (2.0 * p->lambda0 * p->lambda0);
    double q = p->a_ssb / a;
    c->s = q * q * q;
    double chi_bg = c->s < 1.0 ? std::sqrt(1.0 - c->s) : 0.0;
    *ref_scale = c->A * c->s * chi_bg;
    return true;
  }
  if (model == ISIS_FOFR_HS) {
    if (p->n < 1 || p->n > 8 || !(p->fR0_abs > 0)) return false;
    // Sect. 4.2, the non-canonical equation for u with b = e^u
    double r = grid->Omega_L / grid->Omega_m, np1 = p->n + 1.0;
    c->np1 = np1;
    c->inv_np1 = 1.0 / np1;
    c->K1 = grid->Omega_m * a * H02;
    c->K2 = grid->Omega_m * a * a * a * a * H02 * (1.0 + 4.0 * r) * std::pow(p->fR0_abs * a * a, 1.0 / np1);
    c->K3 = grid->Omega_m * a * H02 * (1.0 + 4.0 * a * a * a * r);
    c->fscale = 1.0;  // field form in u itself; the refinement's first phase shifts it
    c->fKx = c->K2;
    c->fK3x = c->K3 - c->K2;
    *ref_scale = c->K1;
    return true;
  }
  if (model == ISIS_CHAMELEON) {
    if (!(p->lambda0 > 0) || !(p->cham_n > -1.0) || !(p->cham_n <= 8.0)) return false;
    // The chameleon equation of Sect. 6 as a free source (Sect. 2), in u = ln(phi / phi_0):
    // div(e^u grad u) = A_c [a^-3 eta - e^{-(1+n) u}], A_c = a^2 / ((1+n) lambda0^2): the f(R) operator with
    // K1 = K3 = A_c a^-3, K2 = A_c and the exponent 1/(n+1) of f(R) replaced by 1+n.
    const double Ac = a * a / ((1.0 + p->cham_n) * p->lambda0 * p->lambda0);
    c->inv_np1 = 1.0 + p->cham_n;
    c->np1 = 1.0 / c->inv_np1;
    c->K1 = Ac / (a * a * a);
    c->K2 = Ac;
    c->K3 = c->K1;
    c->fscale = 1.0;
    c->fKx = c->K2;
    c->fK3x = c->K3 - c->K2;
    *ref_scale = c->K1;
    return true;
  }
  return false;
}

static void fill_common(SolveArgs& A, const isis_grid* g, double a, const void* eta, void* phi, double tol,
                        const isis_mg_opts& o, isis_solve_info* info, void* stream) {
  A.N = g->N;
  A.box = g->box;
  A.a = a;
  A.eta = eta;
  A.phi = phi;
  A.tol = tol;
  A.nu1 = o.nu1;
  A.nu2 = o.nu2;
  A.ncoarse = o.n_coarsest;
  A.max_cycles = o.max_cycles;
  A.inner = o.inner_cycles;
  A.prec = o.prec;
  A.init = o.init;
  A.fmg = o.fmg;
  A.info = info;
  A.st = (cudaStream_t)stream;
  std::memset(&A.coef, 0, sizeof(A.coef));
}

// ---------------------------------------------------------------------------
// Launch counting and event profiling (isis_prof.cuh)
// ---------------------------------------------------------------------------

static const char* kKindNames[KK_COUNT] = {
    "smooth_fine",    "smooth_coarse", "resid_restrict_fine", "resid_restrict_coarse", "coarse_sigma",
    "prolong_fine",   "prolong_coarse", "coarse_newton",      "norm_fine",             "outer_residual64",
    "update64",       "setup",         "reduce",              "init_guess",            "cic_scatter",
    "cic_finish",     "force_grid",    "force_gather",        "unet_conv",             "unet_elem",
    "patch_smooth",   "patch_other",   "patch_coarsest",      "coarse_cycle"};

struct ProfRec {
  int kind;
  int ev;
  double bytes;
};
static bool g_prof_on = false;
static long long g_launches = 0;
static std::vector<cudaEvent_t> g_events;
static int g_next_event = 0;
static int g_pending = -1;
static std::vector<ProfRec> g_recs;

static int take_event() {
  if (g_next_event >= (int)g_events.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return -1;
    g_events.push_back(e);
  }
  return g_next_event++;
}

void prof_pre(cudaStream_t st) {
  g_pending = -1;
  if (!g_prof_on) return;
  int a = take_event();
  if (a < 0) return;
  if (cudaEventRecord(g_events[a], st) != cudaSuccess) return;
  g_pending = a;
}

bool prof_enabled() { return g_prof_on; }
long long prof_launches() { return g_launches; }
void prof_add_launches(long long n) { g_launches += n; }

void prof_post(int kind, double bytes, cudaStream_t st) {
  ++g_launches;
  if (!g_prof_on || g_pending < 0) return;
  int b = take_event();
  if (b < 0 || b != g_pending + 1) return;
  if (cudaEventRecord(g_events[b], st) != cudaSuccess) return;
  g_recs.push_back({kind, g_pending, bytes});
  g_pending = -1;
}

}  // namespace isis

using namespace isis;

extern "C" {

const char* isis_strerror(isis_status s) {
  switch (s) {
    case ISIS_OK: return "ok";
    case ISIS_EINVAL: return "invalid argument";
    case ISIS_ENOCONV: return "no convergence within max_cycles";
    case ISIS_ENAN: return "non-finite residual or singular coarsest Jacobian";
    case ISIS_ECUDA: return "CUDA error";
    case ISIS_ENOMEM: return "device allocation failed";
    case ISIS_ETIMEOUT: return "device wait timed out";
    case ISIS_EINTERNAL: return "internal error";
  }
  return "unknown status";
}

void isis_release_workspace(void) {
  cudaDeviceSynchronize();
  for (Workspace* w : g_ws) free_ws(w);
  g_ws.clear();
  for (auto& d : g_dep) cudaFree(d.acc);
  g_dep.clear();
  for (auto& d : g_fgrid) cudaFree(d.acc);
  g_fgrid.clear();
}

void isis_prof_enable(int on) { g_prof_on = on != 0; }

void isis_prof_reset(void) {
  g_launches = 0;
  g_recs.clear();
  g_next_event = 0;
  g_pending = -1;
}

int64_t isis_launch_count(void) { return g_launches; }

isis_status isis_selftest_exp_ff(const double* x, double* y, int n, void* stream) {
  if (!x || !y || n < 0) return ISIS_EINVAL;
  if (n == 0) return ISIS_OK;
  static float2* tab = nullptr;
  if (!tab) {
    float2 h[64];
    ff_exp_table_fill(h);
    if (cudaMalloc(&tab, sizeof(h)) != cudaSuccess) return ISIS_ENOMEM;
    if (cudaMemcpy(tab, h, sizeof(h), cudaMemcpyHostToDevice) != cudaSuccess) return ISIS_ECUDA;
  }
  cudaStream_t st = (cudaStream_t)stream;
  ISIS_LAUNCH(KK_SETUP, 16.0 * n, st,
              (selftest_exp_ff<<<(unsigned)((n / 2 + 256) / 256), 256, 0, st>>>(x, y, n, tab, ff_exp_consts())));
  return ISIS_OK;
}

isis_status isis_selftest_ff_to_f64(const float* hl, double* out, int n, void* stream) {
  if (!hl || !out || n < 0) return ISIS_EINVAL;
  if (n == 0) return ISIS_OK;
  cudaStream_t st = (cudaStream_t)stream;
  ISIS_LAUNCH(KK_SETUP, 16.0 * n, st,
              (selftest_ff_to_f64<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(hl, out, n)));
  return ISIS_OK;
}

int isis_prof_read(isis_prof_entry* out, int max) {
  cudaDeviceSynchronize();
  constexpr int kAll = KK_COUNT * kKindTags;
  // names "kind" or "kind[model/form]", built once
  static std::vector<std::string> names;
  if (names.empty()) {
    static const char* kTag[kKindTags] = {"", "[poisson/field]", "[poisson/delta]", "[symmetron/field]",
                                          "[symmetron/delta]", "[fofr/field]", "[fofr/delta]"};
    for (int t = 0; t < kKindTags; ++t)
      for (int k = 0; k < KK_COUNT; ++k) names.push_back(std::string(kKindNames[k]) + kTag[t]);
  }
  std::vector<long long> cnt(kAll, 0);
  std::vector<double> ms(kAll, 0.0), by(kAll, 0.0);
  for (const ProfRec& r : g_recs) {
    float t = 0.f;
    if (r.kind < 0 || r.kind >= kAll) continue;
    if (cudaEventElapsedTime(&t, g_events[r.ev], g_events[r.ev + 1]) != cudaSuccess) continue;
    cnt[r.kind] += 1;
    ms[r.kind] += t;
    by[r.kind] += r.bytes;
  }
  cudaGetLastError();
  int n = 0;
  for (int k = 0; k < kAll && n < max; ++k)
    if (cnt[k] > 0) out[n++] = {names[k].c_str(), cnt[k], ms[k], by[k]};
  return n;
}

isis_status isis_poisson_solve(const isis_grid* grid, double a, const void* eta, void* Phi, double tol,
                               const isis_mg_opts* opts, isis_solve_info* info, void* stream) {
  isis_mg_opts o;
  if (!grid_ok(grid) || !eta || !Phi || !(a > 0) || !(tol >= 0) || !opts_resolve(opts, &o, grid->N))
    return ISIS_EINVAL;
  SolveArgs A;
  fill_common(A, grid, a, eta, Phi, tol, o, info, stream);
  // Sect. 3.1: lap Phi = (3/2) Om H0^2 delta / a
  A.coef.KP = 1.5 * grid->Omega_m * grid->H0 * grid->H0 / a;
  A.ref_scale = A.coef.KP;
  return run_poi(A);
}

isis_status isis_scalar_solve(isis_model model, const isis_params* p, const isis_grid* grid, double a,
                              const void* eta, void* phi, double tol, const isis_mg_opts* opts,
                              isis_solve_info* info, void* stream) {
  isis_mg_opts o;
  if (!grid_ok(grid) || !p || !eta || !phi || !(a > 0) || !(tol >= 0) || !opts_resolve(opts, &o, grid->N))
    return ISIS_EINVAL;
  SolveArgs A;
  fill_common(A, grid, a, eta, phi, tol, o, info, stream);
  if (!model_coef(model, p, grid, a, &A.coef, &A.ref_scale)) return ISIS_EINVAL;
  return model == ISIS_SYMMETRON ? run_sym(A) : run_fofr(A);
}

isis_status isis_background_field(isis_model model, const isis_params* p, const isis_grid* grid, double a,
                                  double* out) {
  if (!p || !grid || !out || !(a > 0) || !std::isfinite(a) || !(grid->H0 > 0) || !(grid->Omega_m > 0) ||
      !(grid->Omega_L >= 0))
    return ISIS_EINVAL;
  Coef c;
  double ref_scale = 0.0;
  std::memset(&c, 0, sizeof(c));
  if (!model_coef(model, p, grid, a, &c, &ref_scale)) return ISIS_EINVAL;
  *out = model == ISIS_SYMMETRON ? background_value<SYM>(c) : background_value<FOFR>(c);
  return ISIS_OK;
}

// Refinement patches (Sect. 3.3.1, Sect. 3.4.1).
static isis_status patch_common(PatchArgs& P, const isis_grid* grid, double a, const isis_patch* box,
                                const void* parent, const uint8_t* flags, const void* eta, void* phi, double tol,
                                const isis_mg_opts* opts, isis_solve_info* info, void* stream) {
  if (!grid_ok(grid) || !box || !parent || !flags || !eta || !phi || !(a > 0) || !(tol >= 0)) return ISIS_EINVAL;
  isis_mg_opts o = {2, 2, 4, 100, ISIS_F64, 2, ISIS_INIT_INPUT, 0};
  if (opts) o = *opts;
  if (o.nu1 < 0 || o.nu1 > 16 || o.nu2 < 0 || o.nu2 > 16 || o.max_cycles < 0 || o.max_cycles > 128) return ISIS_EINVAL;
  if ((o.prec != ISIS_F64 && o.prec != ISIS_F32_REFINE64) || (o.init != ISIS_INIT_INPUT && o.init != ISIS_INIT_PARENT))
    return ISIS_EINVAL;
  if (o.prec == ISIS_F32_REFINE64 && (o.inner_cycles < 1 || o.inner_cycles > 16)) return ISIS_EINVAL;
  if (box->level < 1 || box->level > 12) return ISIS_EINVAL;
  int64_t nflag = 0;
  for (int d = 0; d < 3; ++d) {
    const int n = box->n[d], pn = box->parent_dims[d], o0 = box->origin[d];
    if (n < 4 || (n & 1) || n > 2048) return ISIS_EINVAL;
    if (box->parent_periodic) {
      if (box->level != 1 || pn != grid->N || n > pn || o0 < 0 || o0 >= pn) return ISIS_EINVAL;
    } else if (box->level < 2 || pn < 1 || o0 < 1 || o0 + n + 1 > pn) {
      return ISIS_EINVAL;
    }
  }
  // the coarsest patch level is relaxed by one block: keep it small
  {
    int m[3] = {2 * box->n[0], 2 * box->n[1], 2 * box->n[2]};
    while (!(m[0] & 1) && !(m[1] & 1) && !(m[2] & 1) && std::min(m[0], std::min(m[1], m[2])) >= 8) {
      m[0] /= 2; m[1] /= 2; m[2] /= 2;
    }
    if ((int64_t)m[0] * m[1] * m[2] > 32768) return ISIS_EINVAL;
  }
  // refine flags: none on the outer layer of the box; count the unknowns
  const size_t nb = (size_t)box->n[0] * box->n[1] * box->n[2];
  std::vector<uint8_t> hf(nb);
  if (cudaMemcpyAsync(hf.data(), flags, nb, cudaMemcpyDeviceToHost, (cudaStream_t)stream) != cudaSuccess ||
      cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) {
    cudaGetLastError();
    return ISIS_ECUDA;
  }
  for (int i = 0; i < box->n[0]; ++i)
    for (int j = 0; j < box->n[1]; ++j)
      for (int k = 0; k < box->n[2]; ++k) {
        const uint8_t f = hf[((size_t)i * box->n[1] + j) * box->n[2] + k];
        if (!f) continue;
        if (i == 0 || j == 0 || k == 0 || i == box->n[0] - 1 || j == box->n[1] - 1 || k == box->n[2] - 1)
          return ISIS_EINVAL;
        ++nflag;
      }
  std::memset(&P.coef, 0, sizeof(P.coef));
  for (int d = 0; d < 3; ++d) {
    P.n[d] = box->n[d];
    P.origin[d] = box->origin[d];
    P.pn[d] = box->parent_dims[d];
  }
  P.periodic = box->parent_periodic ? 1 : 0;
  P.h = grid->box / ((double)grid->N * (double)(1 << box->level));
  P.parent = (const double*)parent;
  P.flags = flags;
  P.eta = (const double*)eta;
  P.phi = (double*)phi;
  P.unknowns = 8 * nflag;
  P.tol = tol;
  P.nu1 = o.nu1;
  P.nu2 = o.nu2;
  P.max_cycles = o.max_cycles;
  P.prec = o.prec;
  P.inner = o.inner_cycles;
  P.init_parent = o.init == ISIS_INIT_PARENT ? 1 : 0;
  P.info = info;
  P.st = (cudaStream_t)stream;
  P.eref = 1.0;
  return ISIS_OK;
}

isis_status isis_patch_poisson_solve(const isis_grid* grid, double a, const isis_patch* box, const void* parent,
                                     const uint8_t* flags, const void* eta, void* Phi, double tol,
                                     const isis_mg_opts* opts, isis_solve_info* info, void* stream) {
  PatchArgs P;
  isis_status st = patch_common(P, grid, a, box, parent, flags, eta, Phi, tol, opts, info, stream);
  if (st != ISIS_OK) return st;
  if (!std::isfinite(box->eta_mean)) return ISIS_EINVAL;
  P.model = POI;
  P.coef.KP = 1.5 * grid->Omega_m * grid->H0 * grid->H0 / a;
  P.coef.eta_mean = box->eta_mean;
  P.eref = box->eta_mean;
  P.ref_scale = P.coef.KP;
  return run_patch_poi(P);
}

isis_status isis_patch_scalar_solve(isis_model model, const isis_params* params, const isis_grid* grid, double a,
                                    const isis_patch* box, const void* parent, const uint8_t* flags,
                                    const void* eta, void* phi, double tol, const isis_mg_opts* opts,
                                    isis_solve_info* info, void* stream) {
  if (!params) return ISIS_EINVAL;
  PatchArgs P;
  isis_status st = patch_common(P, grid, a, box, parent, flags, eta, phi, tol, opts, info, stream);
  if (st != ISIS_OK) return st;
  if (!model_coef(model, params, grid, a, &P.coef, &P.ref_scale)) return ISIS_EINVAL;
  if (model == ISIS_SYMMETRON) {
    P.model = SYM;
    return run_patch_sym(P);
  }
  P.model = FOFR;
  return run_patch_fofr(P);
}

}  // extern "C"
