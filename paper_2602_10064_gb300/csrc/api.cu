// C-ABI entry points of libtacaw.so (declared in include/tacaw.h): context, host-side FP64
// tables (twiddles, masks, propagator, spreading-kernel transform) and the orchestration of
// the slice and spectrum kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/tacaw.h"
#include "tacaw_api_internal.h"
#include "tacaw_internal.cuh"

using namespace tacaw;

namespace {

// CODATA 2018 constants (h, e, c exact in SI).
constexpr double kH = 6.62607015e-34, kQe = 1.602176634e-19, kMe = 9.1093837015e-31, kC = 299792458.0;
constexpr double kA0 = 0.529177210903, kEps0 = 8.8541878128e-12;

double wavelength_A(double V) {
  const double eV = kQe * V;
  return kH / std::sqrt(2.0 * kMe * eV * (1.0 + eV / (2.0 * kMe * kC * kC))) * 1e10;
}
double sigma_per_VA(double V) {
  const double gamma = 1.0 + kQe * V / (kMe * kC * kC);
  return 2.0 * M_PI * gamma * kMe * kQe * (wavelength_A(V) * 1e-10) / (kH * kH) * 1e-10;
}
double kirkland_pref() { return 2.0 * M_PI * kA0 * (kQe / (4.0 * M_PI * kEps0) * 1e10); }

double kfreq(int i, int n, double L) {
  const int m = (i < (n + 1) / 2) ? i : i - n;
  return (double)m / L;
}

// Circular mask |k|^2 <= kr^2 (kr <= 0: everything inside).
bool in_disc(int iy, int ix, int nx, int ny, double Lx, double Ly, double kr) {
  const double kx = kfreq(ix, nx, Lx), ky = kfreq(iy, ny, Ly);
  const double k2 = kx * kx + ky * ky;
  return k2 <= kr * kr;
}

double band_radius(const tacaw_params& p) {
  if (p.bandlimit <= 0.0) return -1.0;
  const double a = 0.5 * (double)p.nx / p.cell[0], b = 0.5 * (double)p.ny / p.cell[1];
  return p.bandlimit * (a < b ? a : b);
}

// Transform lengths the slice kernels are built for: powers of two 32 .. 1024, 3 * 2^k for
// 96 .. 768, and 1152 = 9 * 2^7.
bool grid_supported(int n) {
  if (n >= 32 && n <= 1024 && (n & (n - 1)) == 0) return true;
  return n == 96 || n == 192 || n == 384 || n == 768 || n == 1152;
}

// Gauss-Legendre nodes and weights on [-1, 1] (Newton on P_n).
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.resize(n);
  w.resize(n);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = 0.0;
      for (int k = 1; k <= n; ++k) {
        const double p2 = p1;
        p1 = p0;
        p0 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p2) / k;
      }
      dp = n * (z * p0 - p1) / (z * z - 1.0);
      const double dz = p0 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

constexpr int kSpreadHalf = 6;         // kernel width w = 12 grid points
constexpr double kSpreadBeta = 24.0;   // beta = 2.0 w

double es_phi(double z) {
  const double a = 1.0 - z * z;
  return a > 0.0 ? std::exp(kSpreadBeta * (std::sqrt(a) - 1.0)) : 0.0;
}

// Phi(m) = h int_{-1}^{1} phi(z) cos(2 pi m h z / N) dz: the transform of the spreading kernel.
double es_transform(int m, int N) {
  static std::vector<double> gx, gw;
  static std::once_flag once;
  std::call_once(once, [] { gauss_legendre(160, gx, gw); });
  double s = 0.0;
  for (size_t i = 0; i < gx.size(); ++i)
    s += gw[i] * es_phi(gx[i]) * std::cos(2.0 * M_PI * m * kSpreadHalf * gx[i] / N);
  return kSpreadHalf * s;
}

}  // namespace

// ===================================================================================
// context
// ===================================================================================
namespace tacaw {

int set_err(tacaw_ctx* c, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  return code;
}

static cudaEvent_t prof_event(tacaw_ctx* c) {
  Profiler& P = c->prof;
  if (P.next == P.pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    P.pool.push_back(e);
  }
  return P.pool[P.next++];
}

ProfScope::ProfScope(tacaw_ctx* c, const char* name, cudaStream_t s, double bytes, double flops) : ctx(c), st(s) {
  if (!c->prof.on) return;
  rec.name = name;
  rec.bytes = bytes;
  rec.flops = flops;
  const auto& sel = c->prof.select;
  if (!sel.empty() && std::find(sel.begin(), sel.end(), name) == sel.end()) {
    c->prof.recs.push_back(rec);  // counted, not timed (no events)
    return;
  }
  rec.a = prof_event(c);
  rec.b = prof_event(c);
  if (!rec.a || !rec.b) return;
  active = cudaEventRecord(rec.a, st) == cudaSuccess;
}

ProfScope::~ProfScope() {
  if (!active) return;
  if (cudaEventRecord(rec.b, st) == cudaSuccess) ctx->prof.recs.push_back(rec);
}

// Results go to page-locked host memory by SM stores by default: right after a run, a copy-engine
// transfer of c4's 8 GiB S into page-locked memory ran at 16-31 GB/s, the SM copy at 193 GB/s.
cudaError_t copy_rows_out(tacaw_ctx* ctx, float* dst, size_t dp, const float* src, size_t sp, size_t width,
                          size_t rows, cudaStream_t st) {
  if (width == 0 || rows == 0) return cudaSuccess;
  cudaPointerAttributes a{};
  const bool known = cudaPointerGetAttributes(&a, dst) == cudaSuccess;
  if (!known) cudaGetLastError();  // pageable memory: not an error
  float* target = nullptr;
  if (known && (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged)) target = dst;
  else if (known && a.type == cudaMemoryTypeHost && ctx->host_copy == 1 && a.devicePointer)
    target = static_cast<float*>(a.devicePointer);
  if (target) return launch_copy_out(src, (int64_t)sp, target, (int64_t)dp, (int64_t)width, (int64_t)rows, st);
  return cudaMemcpy2DAsync(dst, sizeof(float) * dp, src, sizeof(float) * sp, sizeof(float) * width, rows,
                           cudaMemcpyDefault, st);
}

cudaError_t copy_to_host(tacaw_ctx* ctx, float* dst, const float* src, size_t n, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  if (ctx->host_copy == 1) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, dst) == cudaSuccess && a.type == cudaMemoryTypeHost && a.devicePointer)
      return launch_copy_out(src, (int64_t)n, static_cast<float*>(a.devicePointer), (int64_t)n, (int64_t)n, 1, st);
    cudaGetLastError();  // pageable memory: not an error, the copy engine takes it
  }
  return cudaMemcpyAsync(dst, src, sizeof(float) * n, cudaMemcpyDeviceToHost, st);
}

constexpr size_t kStagingBytes = (size_t)32 << 20;

cudaError_t staged_copy(tacaw_ctx* ctx, void* dst, const void* src, size_t bytes, cudaStream_t st) {
  if (bytes == 0) return cudaSuccess;
  PinnedRing& R = ctx->staging;
  const size_t need = (bytes + 255) & ~(size_t)255;
  if (need > kStagingBytes) return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st);
  if (!R.base) {
    const cudaError_t e = cudaMallocHost((void**)&R.base, kStagingBytes);
    if (e != cudaSuccess) return e;
    R.cap = kStagingBytes;
    R.head = 0;
  }
  // retire the regions whose copies have completed (oldest first)
  while (!R.inflight.empty() && cudaEventQuery(R.inflight.front().done) == cudaSuccess) {
    R.free_events.push_back(R.inflight.front().done);
    R.inflight.erase(R.inflight.begin());
  }
  cudaGetLastError();  // a not-ready query is not an error
  size_t off = R.head + need <= R.cap ? R.head : 0;  // wrap to the start when the tail is short
  // wait for (and retire) the in-flight regions that overlap [off, off + need)
  for (size_t i = 0; i < R.inflight.size();) {
    const PinnedRing::Span& sp = R.inflight[i];
    if (sp.off < off + need && off < sp.end) {
      const cudaError_t e = cudaEventSynchronize(sp.done);
      if (e != cudaSuccess) return e;
      R.free_events.push_back(sp.done);
      R.inflight.erase(R.inflight.begin() + (long)i);
    } else {
      ++i;
    }
  }
  std::memcpy(R.base + off, src, bytes);
  cudaError_t e = cudaMemcpyAsync(dst, R.base + off, bytes, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return e;
  cudaEvent_t ev;
  if (!R.free_events.empty()) {
    ev = R.free_events.back();
    R.free_events.pop_back();
  } else if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) {
    return e;
  }
  if ((e = cudaEventRecord(ev, st)) != cudaSuccess) return e;
  R.inflight.push_back({off, off + need, ev});
  R.head = off + need;
  return cudaSuccess;
}

int cuda_err(tacaw_ctx* c, cudaError_t e, const char* where) {
  if (e == cudaSuccess) return TACAW_OK;
  if (e == cudaErrorMemoryAllocation) return set_err(c, TACAW_ENOMEM, "%s: %s", where, cudaGetErrorString(e));
  return set_err(c, TACAW_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

}  // namespace tacaw

#define CK(expr)                                              \
  do {                                                        \
    cudaError_t e_ = (expr);                                  \
    if (e_ != cudaSuccess) return cuda_err(ctx, e_, #expr);   \
  } while (0)

#define TRY_RC(expr)            \
  do {                          \
    int rc_ = (expr);           \
    if (rc_ != TACAW_OK) return rc_; \
  } while (0)

namespace {

template <class T>
int owned_alloc(tacaw_ctx* ctx, T** p, size_t n) {
  void* v = nullptr;
  // stream-ordered on the legacy stream (which non-blocking streams do not wait for): a plain
  // cudaMalloc can wait for the whole device, and tables are built while requests run; the
  // builders synchronise the legacy stream before the tables are used
  cudaError_t e = cudaMallocAsync(&v, sizeof(T) * std::max<size_t>(n, 1), 0);
  if (e != cudaSuccess) return cuda_err(ctx, e, "cudaMalloc");
  ctx->owned.push_back(v);
  *p = static_cast<T*>(v);
  return TACAW_OK;
}

int is_device_ptr(const void* p) {
  if (!p) return 0;
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// The spreading potential resolves the modes |k| <= kbl from the N-point grid, which needs
// the aliases at N - kbl to stay outside the band: kbl <= (2/3) Nyquist (1.5x headroom).
constexpr double kMaxSpreadBandlimit = 2.0 / 3.0 + 1e-12;

int check_spread_band(tacaw_ctx* ctx, const tacaw_params* p) {
  if (!(p->bandlimit > 0.0) || p->bandlimit > kMaxSpreadBandlimit)
    return set_err(ctx, TACAW_EINVAL,
                   "building the potential needs a band limit in (0, 2/3] of Nyquist (got %g): the spread "
                   "structure factor is accurate only inside it", p->bandlimit);
  return TACAW_OK;
}

tacaw_probe default_probe() {
  tacaw_probe p{};
  p.n_probes = 1;
  return p;
}

bool has_aberrations(const tacaw_probe& pr) {
  return pr.defocus != 0.0 || pr.cs_mm != 0.0 || pr.astig != 0.0 || pr.coma != 0.0;
}

int check_params(tacaw_ctx* ctx, const tacaw_params* p) {
  if (!p) return set_err(ctx, TACAW_EINVAL, "params is NULL");
  if (!grid_supported(p->nx) || !grid_supported(p->ny))
    return set_err(ctx, TACAW_EINVAL,
                   "grid %dx%d: nx, ny must be powers of two in [32, 1024] or one of 96, 192, 384, 768, 1152",
                   p->nx, p->ny);
  if (p->n_slices < 1 || p->n_slices > 256) return set_err(ctx, TACAW_EINVAL, "n_slices %d not in [1, 256]", p->n_slices);
  for (int i = 0; i < 3; ++i)
    if (!(p->cell[i] > 0.0) || !std::isfinite(p->cell[i])) return set_err(ctx, TACAW_EINVAL, "cell[%d] must be > 0", i);
  if (!(p->voltage_ev > 0.0)) return set_err(ctx, TACAW_EINVAL, "voltage_ev must be > 0");
  if (p->bandlimit > 0.0 && (p->bandlimit > 1.0 || !std::isfinite(p->bandlimit)))
    return set_err(ctx, TACAW_EINVAL, "bandlimit must be in (0, 1] or <= 0 for none");
  return TACAW_OK;
}

// Band of columns inside a disc of radius kr (kr <= 0: all columns).
void make_band(int nx, int ny, double Lx, double Ly, double kr, int& W, int& Wp, int& mb, std::vector<int>& nb) {
  if (kr <= 0.0 || in_disc(0, nx / 2, nx, ny, Lx, Ly, kr)) {
    W = nx;
    mb = nx / 2;
  } else {
    mb = -1;
    for (int m = 0; m < nx / 2; ++m)
      if (in_disc(0, m, nx, ny, Lx, Ly, kr)) mb = m;
      else break;
    W = mb >= 0 ? 2 * mb + 1 : 0;
  }
  Wp = std::max(32, (W + 31) / 32 * 32);
  if (Wp > nx) Wp = nx;
  nb.assign(Wp, -1);
  for (int c = 0; c < W; ++c) {
    const int x = c <= mb ? c : nx - (W - c);
    int best = -1;
    for (int n = 0; n <= ny / 2; ++n) {
      const int iy = n;  // n = ny/2 is the Nyquist row (index ny/2)
      if (kr <= 0.0 || in_disc(iy, x, nx, ny, Lx, Ly, kr)) best = n;
      else break;
    }
    nb[c] = best;
  }
}

}  // namespace

namespace tacaw {

// Geometry tables for one parameter set (cached).  Requires the form-factor table.
int get_geo(tacaw_ctx* ctx, const tacaw_params& p, GeoCache** out) {
  std::vector<double> key = {(double)p.nx, (double)p.ny, p.cell[0], p.cell[1], p.cell[2], (double)p.n_slices,
                             p.voltage_ev, p.bandlimit};
  auto it = ctx->geos.find(key);
  if (it != ctx->geos.end() && it->second->ff_version == ctx->ff_version) {
    *out = it->second.get();
    return TACAW_OK;
  }
  auto g = std::make_unique<GeoCache>();
  const int nx = p.nx, ny = p.ny;
  const double Lx = p.cell[0], Ly = p.cell[1];
  std::vector<int> nb;
  int W, Wp, mb;
  make_band(nx, ny, Lx, Ly, band_radius(p), W, Wp, mb, nb);
  if (W == 0) return set_err(ctx, TACAW_EINVAL, "band limit excludes every column");
  TRY_RC(owned_alloc(ctx, &g->colnb, Wp));
  CK(cudaMemcpy(g->colnb, nb.data(), sizeof(int) * Wp, cudaMemcpyHostToDevice));
  g->band = Band{W, Wp, mb, g->colnb};
  // propagator P = exp(-i pi lambda dz (kx^2 + ky^2)) = Px Py, FP64 on host
  const double lam = wavelength_A(p.voltage_ev), dz = p.cell[2] / p.n_slices;
  std::vector<float2> hx(Wp, make_float2(0.f, 0.f)), hy(ny);
  for (int c = 0; c < W; ++c) {
    const int x = c <= mb ? c : nx - (W - c);
    const double kx = kfreq(x, nx, Lx), ph = -M_PI * lam * dz * kx * kx;
    hx[c] = make_float2((float)std::cos(ph), (float)std::sin(ph));
  }
  for (int y = 0; y < ny; ++y) {
    const double ky = kfreq(y, ny, Ly), ph = -M_PI * lam * dz * ky * ky;
    hy[y] = make_float2((float)std::cos(ph), (float)std::sin(ph));
  }
  TRY_RC(owned_alloc(ctx, &g->px, Wp));
  TRY_RC(owned_alloc(ctx, &g->py, ny));
  CK(cudaMemcpy(g->px, hx.data(), sizeof(float2) * Wp, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(g->py, hy.data(), sizeof(float2) * ny, cudaMemcpyHostToDevice));
  // spreading-kernel transforms
  std::vector<double> phx(Wp, 1.0), phy(ny);
  for (int c = 0; c < W; ++c) {
    const int x = c <= mb ? c : nx - (W - c);
    phx[c] = es_transform((x < (nx + 1) / 2) ? x : x - nx, nx);
  }
  for (int y = 0; y < ny; ++y) phy[y] = es_transform((y < (ny + 1) / 2) ? y : y - ny, ny);
  TRY_RC(owned_alloc(ctx, &g->phix, Wp));
  TRY_RC(owned_alloc(ctx, &g->phiy, ny));
  CK(cudaMemcpy(g->phix, phx.data(), sizeof(double) * Wp, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(g->phiy, phy.data(), sizeof(double) * ny, cudaMemcpyHostToDevice));
  // in-band q list (ascending q = iy * nx + x)
  std::vector<int32_t> qs;
  for (int y = 0; y < ny; ++y) {
    const int n = (y < (ny + 1) / 2) ? y : y - ny;
    for (int x = 0; x < nx; ++x) {
      const int c = x <= mb ? x : (x >= nx - mb ? x - nx + W : -1);
      if (c >= 0 && c < W && std::abs(n) <= nb[c]) qs.push_back(y * nx + x);
    }
  }
  g->nsel = (int64_t)qs.size();
  TRY_RC(owned_alloc(ctx, &g->qsel, qs.size()));
  CK(cudaMemcpy(g->qsel, qs.data(), sizeof(int32_t) * qs.size(), cudaMemcpyHostToDevice));
  // per-row start and count of the in-band points (the compact exit-wave layout), checked
  // against the position rule the last column pass uses
  std::vector<int2> disc(ny, make_int2(0, 0));
  for (size_t i = 0; i < qs.size(); ++i) disc[qs[i] / nx].y++;
  for (int y = 1; y < ny; ++y) disc[y].x = disc[y - 1].x + disc[y - 1].y;
  for (size_t i = 0; i < qs.size(); ++i) {
    const int y = qs[i] / nx, x = qs[i] % nx;
    const int c = x <= mb ? x : x - nx + W, a = (disc[y].y - 1) >> 1;
    const int j = disc[y].y == nx ? c : (c <= a ? c : c - W + 2 * a + 1);
    if ((int64_t)disc[y].x + j != (int64_t)i)
      return set_err(ctx, TACAW_EINVAL, "internal: in-band layout of row %d is not symmetric", y);
  }
  TRY_RC(owned_alloc(ctx, &g->disc, ny));
  CK(cudaMemcpy(g->disc, disc.data(), sizeof(int2) * ny, cudaMemcpyHostToDevice));
  // potential multiplier table over the loaded species (slot = table index)
  const int nslot = (int)ctx->ffZ.size();
  if (nslot > 0) {
    g->nslot = nslot;
    g->npair = (nslot + 1) / 2;
    TRY_RC(owned_alloc(ctx, &g->coef_slots, 12 * (size_t)nslot));
    CK(cudaMemcpy(g->coef_slots, ctx->ffcoef.data(), sizeof(double) * 12 * nslot, cudaMemcpyHostToDevice));
    TRY_RC(owned_alloc(ctx, &g->mtab, (size_t)g->npair * ny * Wp));
    const Geo geo{nx, ny, ctx->tw};
    CK(launch_build_mtab(geo, g->band, g->npair, nslot, g->coef_slots, g->phix, g->phiy, Lx, Ly,
                         kirkland_pref() / (Lx * Ly), g->mtab, 0));
  }
  // the tables are complete (copies and the table kernel on the legacy stream) before any
  // stream uses them; other streams' work is not waited for
  CK(cudaStreamSynchronize(0));
  g->ff_version = ctx->ff_version;
  *out = g.get();
  ctx->geos[key] = std::move(g);
  return TACAW_OK;
}

// Length-F time twiddles exp(-2 pi i j / F).
int get_time_tw(tacaw_ctx* ctx, int64_t F, float2** out) {
  auto it = ctx->time_tw.find(F);
  if (it != ctx->time_tw.end()) {
    *out = it->second;
    return TACAW_OK;
  }
  std::vector<float2> h(F);
  for (int64_t j = 0; j < F; ++j) {
    const double a = -2.0 * M_PI * (double)j / (double)F;
    h[j] = make_float2((float)std::cos(a), (float)std::sin(a));
  }
  float2* d;
  TRY_RC(owned_alloc(ctx, &d, F));
  CK(cudaMemcpy(d, h.data(), sizeof(float2) * F, cudaMemcpyHostToDevice));
  CK(cudaStreamSynchronize(0));  // the copy has landed before any stream reads the table
  ctx->time_tw[F] = d;
  *out = d;
  return TACAW_OK;
}

}  // namespace tacaw

// ===================================================================================
// entry points
// ===================================================================================
extern "C" {

const char* tacaw_version(void) { return "tacaw-gb300 0.1 (sm_103a)"; }

int tacaw_axes(const tacaw_params* params, int64_t n_frames, double* kx, double* ky, double* f_thz,
               double* sampling) {
  if (!params || params->nx < 1 || params->ny < 1 || n_frames < 1) return TACAW_EINVAL;
  const double Lx = params->cell[0], Ly = params->cell[1], dt_ps = params->dt_fs * 1e-3;
  if (!(Lx > 0.0) || !(Ly > 0.0) || !(dt_ps > 0.0) || !std::isfinite(Lx) || !std::isfinite(Ly) ||
      !std::isfinite(dt_ps))
    return TACAW_EINVAL;
  const int64_t F = n_frames;
  if (kx)
    for (int i = 0; i < params->nx; ++i) kx[i] = kfreq(i, params->nx, Lx);
  if (ky)
    for (int i = 0; i < params->ny; ++i) ky[i] = kfreq(i, params->ny, Ly);
  if (f_thz)
    for (int64_t m = 0; m < F; ++m) f_thz[m] = (double)(m < (F + 1) / 2 ? m : m - F) / ((double)F * dt_ps);
  if (sampling) {
    sampling[0] = 1.0 / Lx;
    sampling[1] = 1.0 / Ly;
    sampling[2] = 0.5 * (double)params->nx / Lx;
    sampling[3] = 0.5 * (double)params->ny / Ly;
    sampling[4] = 1.0 / ((double)F * dt_ps);
    sampling[5] = 0.5 / dt_ps;
  }
  return TACAW_OK;
}

int tacaw_create(tacaw_ctx** out, int32_t device, uint64_t hbm_budget_bytes) {
  if (!out) return TACAW_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return TACAW_EINVAL;
  }
  auto* ctx = new (std::nothrow) tacaw_ctx();
  if (!ctx) return TACAW_ENOMEM;
  ctx->device = device;
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) {
    delete ctx;
    return TACAW_ECUDA;
  }
  size_t fr = 0, tot = 0;
  cudaMemGetInfo(&fr, &tot);
  ctx->budget = hbm_budget_bytes ? hbm_budget_bytes : (uint64_t)(0.9 * (double)fr);
  // keep freed stream-ordered memory in the pool between calls
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  // FFT twiddle tables, FP64 on host: exp(-2 pi i j / N) at tw_offset(N) + j
  std::vector<float2> tw(kTwiddleEntries, make_float2(0.f, 0.f));
  std::vector<int> lengths;
  for (int N = 2; N <= 2048; N *= 2) lengths.push_back(N);
  for (int N : kTwiddleOtherLengths) lengths.push_back(N);
  for (int N : lengths)
    for (int j = 0; j < N; ++j) {
      const double a = -2.0 * M_PI * (double)j / (double)N;
      tw[tw_offset(N) + j] = make_float2((float)std::cos(a), (float)std::sin(a));
    }
  if (owned_alloc(ctx, &ctx->tw, tw.size()) != TACAW_OK ||
      cudaMemcpy(ctx->tw, tw.data(), sizeof(float2) * tw.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      owned_alloc(ctx, &ctx->d_status, 1) != TACAW_OK || cudaMemset(ctx->d_status, 0, sizeof(int)) != cudaSuccess ||
      owned_alloc(ctx, &ctx->d_zslot, 256) != TACAW_OK || cudaMemset(ctx->d_zslot, 0xff, 256) != cudaSuccess ||
      cudaDeviceSynchronize() != cudaSuccess) {
    for (void* p : ctx->owned) cudaFree(p);
    delete ctx;
    return TACAW_ECUDA;
  }
  *out = ctx;
  return TACAW_OK;
}

int tacaw_destroy(tacaw_ctx* ctx) {
  if (!ctx) return TACAW_EINVAL;
  cudaSetDevice(ctx->device);
  serving_shutdown(ctx);
  cudaDeviceSynchronize();
  for (auto& sp : ctx->staging.inflight) cudaEventDestroy(sp.done);
  for (cudaEvent_t ev : ctx->staging.free_events) cudaEventDestroy(ev);
  if (ctx->staging.base) cudaFreeHost(ctx->staging.base);
  for (void* p : ctx->owned) cudaFree(p);
  delete ctx;
  return TACAW_OK;
}

const char* tacaw_last_error(const tacaw_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int tacaw_load_form_factors(tacaw_ctx* ctx, const int32_t* Z, const double* coef, int32_t nZ) {
  if (!ctx) return TACAW_EINVAL;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  if (!Z || !coef || nZ < 1 || nZ > 64) return set_err(ctx, TACAW_EINVAL, "nZ must be in [1, 64]");
  for (int i = 0; i < nZ; ++i) {
    for (int j = 0; j < i; ++j)
      if (Z[i] == Z[j]) return set_err(ctx, TACAW_EINVAL, "Z=%d appears twice", Z[i]);
    for (int k = 0; k < 3; ++k)
      if (!(coef[12 * i + 2 * k + 1] > 0.0)) return set_err(ctx, TACAW_EINVAL, "b_%d of Z=%d must be > 0", k + 1, Z[i]);
    for (int k = 0; k < 12; ++k)
      if (!std::isfinite(coef[12 * i + k])) return set_err(ctx, TACAW_EINVAL, "non-finite coefficient");
  }
  for (int i = 0; i < nZ; ++i)
    if (Z[i] < 1 || Z[i] > 255) return set_err(ctx, TACAW_EINVAL, "Z=%d outside [1, 255]", Z[i]);
  std::vector<int8_t> lut(256, -1);
  for (int i = 0; i < nZ; ++i) lut[Z[i]] = (int8_t)i;
  CK(cudaSetDevice(ctx->device));
  CK(cudaMemcpy(ctx->d_zslot, lut.data(), 256, cudaMemcpyHostToDevice));
  CK(cudaStreamSynchronize(0));  // the table has landed before any stream reads it
  ctx->ffZ.assign(Z, Z + nZ);
  ctx->ffcoef.assign(coef, coef + 12 * (size_t)nZ);
  ctx->ff_version++;
  return TACAW_OK;
}

}  // extern "C"

namespace tacaw {

// Slot (form-factor table index) of every atom; host Z in, device int8 out.
// Form-factor slot of every atom.  Z on the device with device_check: mapped on the device, an
// unknown species reported through the status word (tacaw_check), so the host never waits
// for the stream.  Otherwise Z is checked on the host and an unknown species is EINVAL here.
int make_slots(tacaw_ctx* ctx, const int32_t* Z, int64_t A, bool z_on_device, bool device_check, Scratch& sc,
               int8_t** d_slot) {
  if (z_on_device && device_check) {
    CK(sc.get(d_slot, std::max<int64_t>(A, 1)));
    ProfScope ps(ctx, "map_slots", sc.st, (double)A * 5, 0);
    CK(launch_map_slots(Z, A, ctx->d_zslot, *d_slot, ctx->d_status, sc.st));
    return TACAW_OK;
  }
  std::vector<int32_t> hz(A);
  if (A > 0) {
    if (z_on_device) {
      CK(cudaMemcpyAsync(hz.data(), Z, sizeof(int32_t) * A, cudaMemcpyDeviceToHost, sc.st));
      CK(cudaStreamSynchronize(sc.st));
    } else {
      std::memcpy(hz.data(), Z, sizeof(int32_t) * A);
    }
  }
  std::vector<int8_t> hs(A);
  for (int64_t j = 0; j < A; ++j) {
    int s = -1;
    for (size_t i = 0; i < ctx->ffZ.size(); ++i)
      if (ctx->ffZ[i] == hz[j]) s = (int)i;
    if (s < 0) return set_err(ctx, TACAW_EINVAL, "atom %lld has Z=%d, not in the form-factor table", (long long)j, hz[j]);
    hs[j] = (int8_t)s;
  }
  CK(sc.get(d_slot, A));
  if (A > 0) {
    // through the pinned ring: asynchronous, and hs may go out of scope at once
    CK(staged_copy(ctx, *d_slot, hs.data(), A, sc.st));
  }
  return TACAW_OK;
}

// Binned atoms of frames [0, nf): per-(frame, slice) lists, then the row-sorted copy with the
// offsets of every block of SPREAD_YB grid rows that the spreading pass reads.
struct Binned {
  AtomRec* rrecs = nullptr;
  int* boffs = nullptr;
};
int bin_frames(tacaw_ctx* ctx, const tacaw_params& p, const float* pos, const int8_t* slots, int64_t A, int64_t nf,
               Scratch& sc, Binned* out) {
  const int S = p.n_slices, ny = p.ny, nyb = ny / SPREAD_YB;
  AtomRec* recs;
  int* offs;
  CK(sc.get(&recs, (size_t)nf * std::max<int64_t>(A, 1)));
  CK(sc.get(&offs, (size_t)nf * (S + 1)));
  {
    NvtxRange r_bin("binning");
    ProfScope ps(ctx, "bin", sc.st, (double)nf * A * 28, 0);
    CK(launch_bin(pos, A, nf, S, p.cell[0], p.cell[1], p.cell[2], p.nx, p.ny, slots, recs, offs, nullptr, sc.st));
  }
  CK(sc.get(&out->rrecs, (size_t)nf * std::max<int64_t>(A, 1)));
  CK(sc.get(&out->boffs, (size_t)nf * S * (nyb + 1)));
  {
    NvtxRange r_sort("binning_rows");
    ProfScope ps(ctx, "sort_rows", sc.st, (double)nf * A * 48 + (double)nf * S * (nyb + 1) * 4, 0);
    CK(launch_sort_rows(recs, offs, A, nf, S, ny, out->rrecs, out->boffs, sc.st));
  }
  return TACAW_OK;
}

// Potential of slices [s0, s0 + sbc) of frames [f0, f0 + nfc): the spreading row pass into Bp
// and the column pass into Ap [nfc][sbc][ny][Wp] (compact columns), for a row pass out of it.
int potential_block(tacaw_ctx* ctx, const tacaw_params& p, GeoCache* g, const Binned& bn, int64_t A, int64_t f0,
                    int nfc, int s0, int sbc, float2* Bp, float2* Ap, cudaStream_t st) {
  const int S = p.n_slices, ny = p.ny, nyb = ny / SPREAD_YB, nfs = nfc * sbc;
  const Geo geo{p.nx, p.ny, ctx->tw};
  const SpreadKernel sk{kSpreadHalf, (float)kSpreadBeta};
  const double W8 = (double)g->band.W * 8.0, fx = 5.0 * p.nx * std::log2((double)p.nx),
               fy = 5.0 * ny * std::log2((double)ny);
  NvtxRange r_pot("potential");
  {
    ProfScope ps(ctx, "splat_row", st, (double)nfc * A * 16 * sbc / S + (double)nfs * g->npair * ny * W8,
                 (double)nfs * g->npair * ny * fx);
    CK(launch_splat_row(geo, g->band, bn.rrecs + (size_t)f0 * A, bn.boffs + (size_t)f0 * S * (nyb + 1), A, S, s0,
                        sbc, nfs, g->npair, sk, Bp, (int)ctx->static_band, st));
  }
  {
    ProfScope ps(ctx, "col_pot", st, (double)nfs * (g->npair + 1) * ny * W8 + (double)g->npair * ny * W8,
                 (double)nfs * (g->npair + 1) * g->band.W * fy);
    CK(launch_col_pot(geo, g->band, Bp, g->mtab, g->npair, nfs, Ap, (int)ctx->static_band, st));
  }
  return TACAW_OK;
}

// Potential of frames [0, nf): binning, then per chunk of `chunk` frames and per block of `sb`
// slices the spreading row pass and the column pass.  Leaves Ap [nfc][sbc][ny][Wp] to
// `sink(f0, nfc, s0, sbc, Ap)`, which runs the row pass out of the potential.
template <class Sink>
int potential_chunks(tacaw_ctx* ctx, const tacaw_params& p, GeoCache* g, const float* pos, const int8_t* slots,
                     int64_t A, int64_t nf, int64_t chunk, int sb, Scratch& sc, Sink sink) {
  const int S = p.n_slices;
  Binned bn;
  TRY_RC(bin_frames(ctx, p, pos, slots, A, nf, sc, &bn));
  float2 *Bp, *Ap;
  const size_t plane = (size_t)p.ny * g->band.Wp;
  CK(sc.get(&Bp, (size_t)chunk * sb * g->npair * plane));
  CK(sc.get(&Ap, (size_t)chunk * sb * plane));
  for (int64_t f0 = 0; f0 < nf; f0 += chunk) {
    const int nfc = (int)std::min<int64_t>(chunk, nf - f0);
    for (int s0 = 0; s0 < S; s0 += sb) {
      const int sbc = std::min(sb, S - s0);
      TRY_RC(potential_block(ctx, p, g, bn, A, f0, nfc, s0, sbc, Bp, Ap, sc.st));
      TRY_RC(sink(f0, nfc, s0, sbc, Ap));
    }
  }
  return TACAW_OK;
}

// Frames per chunk so that `per_frame` bytes of scratch stay under `cap`.
int64_t chunk_frames(int64_t nf, size_t per_frame, size_t cap) {
  int64_t c = (int64_t)std::max<size_t>(1, cap / std::max<size_t>(per_frame, 1));
  return std::min<int64_t>(c, nf);
}

// Band-limited transmission of nfs slices from Ap (potential column-pass output) or V.
// With `compact` (and the transmission band limit on) it stops after the column pass and
// leaves the compact At [nfs][ny][Wp] in t, for the fused slice row pass; otherwise t is the
// full [nfs][ny][nx] transmission function.
bool use_compact_t(const tacaw_params& p, int P) {
  return P == 1 && p.bandlimit_transmission && p.bandlimit > 0.0;
}

// Intermediates of the transmission band limit for up to `nfs` slices, allocated once per call.
struct TransBufs {
  float2* Bt = nullptr;
  float2* At = nullptr;
};
int trans_bufs(tacaw_ctx* ctx, const tacaw_params& p, GeoCache* g, int64_t nfs, bool compact, Scratch& sc,
               TransBufs* tb) {
  if (!(p.bandlimit_transmission && p.bandlimit > 0.0)) return TACAW_OK;
  const size_t plane = (size_t)p.ny * g->band.Wp;
  CK(sc.get(&tb->Bt, (size_t)nfs * plane));
  if (!compact) CK(sc.get(&tb->At, (size_t)nfs * plane));
  return TACAW_OK;
}

int transmission_from(tacaw_ctx* ctx, const tacaw_params& p, GeoCache* g, const float2* Ap, const float* V, int nfs,
                      float2* t, Scratch& sc, const TransBufs& tb, bool compact = false) {
  const Geo geo{p.nx, p.ny, ctx->tw};
  const float sig = (float)sigma_per_VA(p.voltage_ev);
  const int bl = p.bandlimit_transmission && p.bandlimit > 0.0;
  const double W8 = (double)g->band.W * 8.0, row = (double)nfs * p.ny, fx = 5.0 * p.nx * std::log2((double)p.nx),
               fy = 5.0 * p.ny * std::log2((double)p.ny);
  if (!bl) {
    if (Ap) {
      ProfScope ps(ctx, "row_pot_t", sc.st, row * (W8 + 8.0 * p.nx), row * fx);
      CK(launch_row_pot_out(geo, g->band, Ap, nfs, 2, sig, nullptr, t, (int)ctx->static_band, sc.st));
    } else {
      ProfScope ps(ctx, "row_vt", sc.st, row * 12.0 * p.nx, 0);
      CK(launch_row_vt(geo, g->band, V, nfs, 0, sig, t, sc.st));
    }
    return TACAW_OK;
  }
  float2* Bt = tb.Bt;
  float2* At = compact ? t : tb.At;
  if (Ap) {
    ProfScope ps(ctx, "row_pot_t", sc.st, row * 2 * W8, row * 2 * fx);
    CK(launch_row_pot_out(geo, g->band, Ap, nfs, 1, sig, nullptr, Bt, (int)ctx->static_band, sc.st));
  } else {
    ProfScope ps(ctx, "row_vt", sc.st, row * (4.0 * p.nx + W8), row * fx);
    CK(launch_row_vt(geo, g->band, V, nfs, 1, sig, Bt, sc.st));
  }
  {
    ProfScope ps(ctx, "col_t", sc.st, 2.0 * nfs * p.ny * W8, 2.0 * nfs * g->band.W * fy);
    CK(launch_col_t(geo, g->band, Bt, nfs, 1.0f / ((float)p.nx * (float)p.ny), At, (int)ctx->static_band,
                    sc.st));
  }
  if (!compact) {
    ProfScope ps(ctx, "row_tout", sc.st, row * (W8 + 8.0 * p.nx), row * fx);
    CK(launch_row_tout(geo, g->band, At, nfs, t, sc.st));
  }
  return TACAW_OK;
}

// Initial waves psi0[P][ny][nx] for a convergent probe.
int build_probes(tacaw_ctx* ctx, const tacaw_params& p, const tacaw_probe& pr, Scratch& sc, float2** psi0) {
  const int nx = p.nx, ny = p.ny, P = pr.n_probes;
  const double Lx = p.cell[0], Ly = p.cell[1];
  const double kmax = pr.alpha_mrad * 1e-3 / wavelength_A(p.voltage_ev);
  int W, Wp, mb;
  std::vector<int> nb;
  make_band(nx, ny, Lx, Ly, kmax, W, Wp, mb, nb);
  if (W == 0) return set_err(ctx, TACAW_EINVAL, "probe aperture holds no k point");
  int64_t count = 0;
  for (int c = 0; c < W; ++c) count += nb[c] < 0 ? 0 : (nb[c] >= ny / 2 ? ny : 2 * nb[c] + 1);
  std::vector<float2> ex((size_t)P * Wp, make_float2(0.f, 0.f)), ey((size_t)P * ny);
  for (int ip = 0; ip < P; ++ip) {
    const double xp = pr.xy ? pr.xy[2 * ip] : 0.0, yp = pr.xy ? pr.xy[2 * ip + 1] : 0.0;
    for (int c = 0; c < W; ++c) {
      const int x = c <= mb ? c : nx - (W - c);
      const double a = -2.0 * M_PI * kfreq(x, nx, Lx) * xp;
      ex[(size_t)ip * Wp + c] = make_float2((float)std::cos(a), (float)std::sin(a));
    }
    for (int y = 0; y < ny; ++y) {
      const double a = -2.0 * M_PI * kfreq(y, ny, Ly) * yp;
      ey[(size_t)ip * ny + y] = make_float2((float)std::cos(a), (float)std::sin(a));
    }
  }
  // aberration phase exp(-i chi(k)) over the aperture columns, FP64 on the host
  std::vector<float2> chi;
  if (has_aberrations(pr)) {
    const double lam = wavelength_A(p.voltage_ev), cs = pr.cs_mm * 1e7;
    chi.assign((size_t)ny * Wp, make_float2(0.f, 0.f));
    for (int c = 0; c < W; ++c) {
      const int x = c <= mb ? c : nx - (W - c);
      const double kx = kfreq(x, nx, Lx);
      for (int y = 0; y < ny; ++y) {
        const double ky = kfreq(y, ny, Ly), k2 = kx * kx + ky * ky, phk = std::atan2(ky, kx);
        const double ph = M_PI * lam * k2 * (pr.defocus + pr.astig * std::cos(2.0 * (phk - pr.astig_angle))) +
                          (2.0 * M_PI / 3.0) * pr.coma * lam * lam * k2 * std::sqrt(k2) * std::cos(phk - pr.coma_angle) +
                          0.5 * M_PI * cs * lam * lam * lam * k2 * k2;
        chi[(size_t)y * Wp + c] = make_float2((float)std::cos(ph), (float)-std::sin(ph));
      }
    }
  }
  int* d_nb;
  float2 *d_ex, *d_ey, *Bpr, *d_chi = nullptr;
  if (!chi.empty()) {
    CK(sc.get(&d_chi, chi.size()));
    CK(staged_copy(ctx, d_chi, chi.data(), sizeof(float2) * chi.size(), sc.st));
  }
  CK(sc.get(&d_nb, Wp));
  CK(sc.get(&d_ex, ex.size()));
  CK(sc.get(&d_ey, ey.size()));
  CK(sc.get(&Bpr, (size_t)P * ny * Wp));
  CK(sc.get(psi0, (size_t)P * ny * nx));
  CK(staged_copy(ctx, d_nb, nb.data(), sizeof(int) * Wp, sc.st));
  CK(staged_copy(ctx, d_ex, ex.data(), sizeof(float2) * ex.size(), sc.st));
  CK(staged_copy(ctx, d_ey, ey.data(), sizeof(float2) * ey.size(), sc.st));
  const Band ap{W, Wp, mb, d_nb};
  const Geo geo{nx, ny, ctx->tw};
  {
    ProfScope ps(ctx, "probe_col", sc.st, (double)P * ny * Wp * 8, (double)P * W * 5.0 * ny * std::log2((double)ny));
    CK(launch_probe_col(geo, ap, d_ex, d_ey, d_chi, P, (float)(1.0 / std::sqrt((double)count)), Bpr, sc.st));
  }
  {
    ProfScope ps(ctx, "probe_row", sc.st, (double)P * ny * (Wp + nx) * 8, (double)P * ny * 5.0 * nx * std::log2((double)nx));
    CK(launch_probe_row(geo, ap, Bpr, P, (float)(1.0 / std::sqrt((double)nx * ny)), *psi0, sc.st));
  }
  return TACAW_OK;
}

// Slices [s0, s0 + sb) of the multislice of nfc frames.  The transmission function of frame fl
// and slice s is t[fl][s - t_first][ny][nx] of a buffer holding t_slices slices per frame (or
// the compact [..][ny][Wp] with `tfused`).  The waves carry over in Apsi between calls, and the
// exit waves go to psi_k[p][f0 + fl] of a [P][F_total] stack when the block holds the last
// slice: full [ny][nx] planes (zeroed by the caller) or, with `compact`, the nsel in-band
// points of each wave.
int slices(tacaw_ctx* ctx, const tacaw_params& p, GeoCache* g, const float2* t, int t_slices, int t_first, int nfc,
           int s0, int sb, int P, const float2* psi0, int64_t F_total, int64_t f0, float2* psi_k, bool compact,
           Scratch& sc, float2* Apsi, float2* Bpsi, bool tfused) {
  const Geo geo{p.nx, p.ny, ctx->tw};
  const int S = p.n_slices;
  const float nq = (float)p.nx * (float)p.ny;
  const float plane_amp = (float)(1.0 / std::sqrt((double)p.nx * p.ny));
  const double W8 = (double)g->band.W * 8.0, rows = (double)P * nfc * p.ny,
               fx = 5.0 * p.nx * std::log2((double)p.nx), fy = 5.0 * p.ny * std::log2((double)p.ny);
  for (int s = s0; s < s0 + sb; ++s) {
    const bool last = s == S - 1;
    {
      const double in = s > 0 ? W8 : (psi0 ? 8.0 * p.nx : 0.0), tin = tfused ? W8 : 8.0 * p.nx;
      ProfScope ps(ctx, "slice_row", sc.st, rows * (in + tin + W8), rows * ((s > 0 ? 2 : 1) + (tfused ? 1 : 0)) * fx);
      CK(launch_slice_row(geo, g->band, s == 0, psi0 == nullptr, tfused, Apsi, psi0, t, t_slices, s - t_first, P,
                          nfc, plane_amp, Bpsi, (int)ctx->static_band, sc.st));
    }
    {
      const double out = last && compact ? (double)g->nsel * 8.0 * P * nfc : rows * W8;
      ProfScope ps(ctx, "slice_col", sc.st, rows * W8 + out, (double)P * nfc * g->band.W * (last ? 1 : 2) * fy);
      CK(launch_slice_col(geo, g->band, last, Bpsi, g->px, g->py,
                          last ? (float)(1.0 / std::sqrt((double)p.nx * p.ny)) : 1.0f / nq, P, nfc, F_total, f0,
                          compact ? g->disc : nullptr, g->nsel, Apsi, psi_k, (int)ctx->static_band, sc.st));
    }
  }
  return TACAW_OK;
}

// Argument checks shared by tacaw_run and tacaw_submit.
int check_run(tacaw_ctx* ctx, const tacaw_params* params, const tacaw_probe& pr, const float* pos,
              const int32_t* Z, int64_t n_atoms, int64_t n_frames, int32_t precision, int32_t reduce,
              const float* S_out, bool buffers) {
  TRY_RC(check_params(ctx, params));
  if (n_atoms < 0 || n_frames < 1 || pr.n_probes < 1) return set_err(ctx, TACAW_EINVAL, "bad sizes");
  if (n_frames > 65535 || pr.n_probes > 65535) return set_err(ctx, TACAW_EINVAL, "frames and probes must be <= 65535");
  if (pr.alpha_mrad <= 0.0 && !pr.psi0 && pr.n_probes != 1)
    return set_err(ctx, TACAW_EINVAL, "a plane wave takes exactly one probe");
  if (pr.psi0 && !is_device_ptr(pr.psi0)) return set_err(ctx, TACAW_EINVAL, "probe psi0 must be a device pointer");
  TRY_RC(check_spread_band(ctx, params));
  if (ctx->ffZ.empty()) return set_err(ctx, TACAW_EINVAL, "no form-factor table loaded");
  if (buffers && !pos && n_atoms > 0) return set_err(ctx, TACAW_EINVAL, "pos is NULL");
  if (buffers && (!S_out || (!Z && n_atoms > 0))) return set_err(ctx, TACAW_EINVAL, "Z, S_out must not be NULL");
  if (reduce != TACAW_REDUCE_NONE && reduce != TACAW_REDUCE_DETECTOR) return set_err(ctx, TACAW_EINVAL, "bad reduce");
  if (precision < TACAW_DFT_FP32 || precision > TACAW_DFT_TF32) return set_err(ctx, TACAW_EINVAL, "bad precision");
  return TACAW_OK;
}

// Tiling of a run: frames per chunk and slices per block.  A chunk's scratch stays under
// 2 GB; the slice block shrinks below S only when that is what lets one slice launch hold at
// least kMinWaveRows wave rows (several waves of CTAs on every SM), so that the number of
// waves per launch does not fall with the slice count or the grid size.  P is the number of
// probes propagated together (one probe block).
constexpr int64_t kMinWaveRows = 65536;  // default of the "min_wave_rows" option
constexpr size_t kChunkCap = (size_t)2 << 30;
struct RunTiling {
  int64_t chunk;
  int sb;
};
RunTiling run_tiling(const tacaw_ctx* ctx, const tacaw_params& p, const GeoCache* g, int P, int64_t F) {
  const size_t nq = (size_t)p.nx * p.ny, plane = (size_t)p.ny * g->band.Wp, cap = kChunkCap;
  const int S = p.n_slices;
  const size_t per_slice = nq * 8 + plane * 8 * (g->npair + 3), wave = (size_t)P * plane * 16;
  const int64_t rows = ctx->min_wave_rows > 0 ? ctx->min_wave_rows : kMinWaveRows;
  int64_t want = std::min<int64_t>(F, (rows + (int64_t)P * p.ny - 1) / ((int64_t)P * p.ny));
  if (ctx->max_chunk_frames > 0) want = std::min<int64_t>(want, ctx->max_chunk_frames);
  int sb = S;
  if ((size_t)want * (S * per_slice + wave) > cap) {
    const size_t room = cap / (size_t)want;
    sb = room > wave ? (int)std::min<size_t>(S, std::max<size_t>(1, (room - wave) / per_slice)) : 1;
  }
  if (ctx->max_slice_block > 0) sb = (int)std::min<int64_t>(sb, ctx->max_slice_block);
  int64_t c = chunk_frames(F, sb * per_slice + wave, cap);
  if (ctx->max_chunk_frames > 0) c = std::min<int64_t>(c, ctx->max_chunk_frames);
  return RunTiling{c, sb};
}

// Probe blocks of a run.  Every probe needs its exit-wave stack (F in-band points, compact)
// and the time transform's operands until its block is transformed; probes are therefore
// propagated and transformed in blocks of Pb, sized so that a run's scratch stays under the
// context's "max_run_bytes" (default: half the serving budget, at most 64 GiB).  When there is
// more than one block and the transmission functions of the whole trajectory fit a quarter of
// that bound, they are built once and kept; otherwise every block rebuilds them.
struct RunPlan {
  int Pb = 1;         // probes per block
  int nblocks = 1;
  bool keep_t = false;
  bool tf = false;    // compact transmission functions, inverse-transformed by the row pass
  RunTiling rt{1, 1};
};

double spectrum_bytes_per_probe(const GeoCache* g, int64_t F, int32_t precision, int32_t reduce) {
  const double nsel = (double)g->nsel;
  double b = nsel * 16;  // mean
  if (precision == TACAW_DFT_FP32) {
    b += (double)F * nsel * 8;                                    // residual
    if (reduce == TACAW_REDUCE_DETECTOR) b += (double)F * nsel * 4;  // compact S
  } else {
    const double esz = (precision == TACAW_DFT_TF32X3 || precision == TACAW_DFT_TF32) ? 4 : 2;
    const double cpp = std::ceil(nsel / 256.0) * 256.0, kpad = std::ceil(2.0 * F / 64.0) * 64.0 + 32;
    b += cpp * kpad * esz * 2;                                               // B_hi, B_lo
    if (reduce == TACAW_REDUCE_DETECTOR) b += cpp / 256.0 * (double)F * 8;  // tile partial sums
  }
  return b;
}

uint64_t run_cap(const tacaw_ctx* ctx) {
  if (ctx->max_run_bytes > 0) return (uint64_t)ctx->max_run_bytes;
  return std::min<uint64_t>(ctx->budget / 2, (uint64_t)64 << 30);
}

// R trajectories of F frames each can run together, stacked along the frame axis (R F frames
// through the multislice; R time transforms of F frames per probe).
RunPlan run_plan(const tacaw_ctx* ctx, const tacaw_params& p, const GeoCache* g, int P, int64_t Fr, int64_t A,
                 int32_t precision, int32_t reduce, int R) {
  RunPlan pl;
  const int64_t F = Fr * R;  // frames through the multislice
  const double nq = (double)p.nx * p.ny, plane = (double)p.ny * g->band.Wp, S = p.n_slices;
  const double fixed = (double)F * A * 44 + (double)F * (S + 1) * 4 + (double)F * S * (p.ny / SPREAD_YB + 1) * 4;
  const double per_probe = nq * 8 + plane * 8 + (double)F * g->nsel * 8 +
                           R * spectrum_bytes_per_probe(g, Fr, precision, reduce);
  const double cap = (double)run_cap(ctx);
  double room = cap - fixed - 2.0 * (double)kChunkCap;
  int64_t pb = room > per_probe ? (int64_t)(room / per_probe) : 1;
  if (ctx->max_probe_block > 0) pb = std::min<int64_t>(pb, ctx->max_probe_block);
  pb = std::max<int64_t>(1, std::min<int64_t>(pb, P));
  pl.nblocks = (int)((P + pb - 1) / pb);
  pl.Pb = (int)((P + pl.nblocks - 1) / pl.nblocks);  // even blocks
  pl.tf = use_compact_t(p, pl.Pb);
  pl.keep_t = pl.nblocks > 1 && (double)F * S * (pl.tf ? plane : nq) * 8 <= 0.25 * cap;
  pl.rt = run_tiling(ctx, p, g, pl.Pb, F);
  if (pl.keep_t) {
    // the kept t is laid out [F][S]: every chunk builds all its slices at once
    pl.rt.sb = p.n_slices;
    const size_t per_frame = (size_t)S * plane * 8 * (g->npair + 2) + (size_t)pl.Pb * plane * 16;
    pl.rt.chunk = std::min<int64_t>(pl.rt.chunk, chunk_frames(F, per_frame, kChunkCap));
  }
  return pl;
}

// Device bytes a run allocates from the stream-ordered pool (tables cached in the context
// are not counted), mirroring run_impl; used to admit serving requests.
uint64_t run_footprint(tacaw_ctx* ctx, const tacaw_params& p, int P, int64_t Fr, int64_t A, int32_t precision,
                       int32_t reduce, GeoCache* g, int R) {
  const RunPlan pl = run_plan(ctx, p, g, P, Fr, A, precision, reduce, R);
  const int64_t F = Fr * R;
  const double nq = (double)p.nx * p.ny, plane = (double)p.ny * g->band.Wp, S = p.n_slices;
  const double chunk = (double)pl.rt.chunk, sb = pl.rt.sb, Pb = pl.Pb;
  const double tsz = (pl.tf ? plane : nq) * 8;
  double b = 0;
  b += (double)F * A * (12 + 16 + 16) + (double)F * (S + 1) * 4 + A;  // positions, records (binned, row-sorted), slots
  b += (double)F * S * (p.ny / SPREAD_YB + 1) * 4;                      // row-block offsets
  b += chunk * sb * plane * 8 * (g->npair + 2);                         // Bp, Ap, Bt
  if (!pl.tf) b += chunk * sb * plane * 8;                              // At
  b += pl.keep_t ? (double)F * S * tsz : chunk * sb * tsz;             // t
  b += chunk * Pb * plane * 16;                                         // Apsi, Bpsi
  b += Pb * (nq * 8 + plane * 8);                                       // probes (and their column pass)
  b += Pb * (double)F * g->nsel * 8;                                    // compact exit waves
  b += Pb * R * spectrum_bytes_per_probe(g, Fr, precision, reduce);
  return (uint64_t)(b * 1.05) + ((uint64_t)64 << 20);
}

// The whole path on device buffers, stream-ordered: positions d_pos [R Fr][A][3] (device: R
// trajectories of Fr frames, one after the other), Z (host or device), S into d_S (device,
// [P][R][Fr][ny][nx] or [P][R][Fr]).  Scratch comes from the stream-ordered pool.  Probes run
// in blocks (RunPlan): each block's waves are propagated through every frame, their compact
// exit-wave stack is transformed (one transform of Fr frames per probe and trajectory: the
// stack [Pb][R Fr][n_sel] is [Pb R][Fr][n_sel]), and the block's scratch is released before
// the next.
int run_impl(tacaw_ctx* ctx, const tacaw_params& p, const tacaw_probe& pr, const float* d_pos, const int32_t* Z,
             bool z_dev, int64_t A, int64_t Fr, int32_t precision, int32_t reduce, float* d_S, cudaStream_t st,
             int R) {
  const int64_t F = Fr * R;
  GeoCache* g;
  TRY_RC(get_geo(ctx, p, &g));
  Scratch sc(st);
  const int P = pr.n_probes, S = p.n_slices;
  const size_t nq = (size_t)p.nx * p.ny, plane = (size_t)p.ny * g->band.Wp;
  const RunPlan pl = run_plan(ctx, p, g, P, Fr, A, precision, reduce, R);
  const RunTiling rt = pl.rt;
  const size_t tsz = pl.tf ? plane : nq;
  int8_t* slots;
  TRY_RC(make_slots(ctx, Z, A, z_dev, true, sc, &slots));
  Binned bn;
  TRY_RC(bin_frames(ctx, p, d_pos, slots, A, F, sc, &bn));
  float2 *Bp, *Ap, *t;
  CK(sc.get(&Bp, (size_t)rt.chunk * rt.sb * g->npair * plane));
  CK(sc.get(&Ap, (size_t)rt.chunk * rt.sb * plane));
  CK(sc.get(&t, pl.keep_t ? (size_t)F * S * tsz : (size_t)rt.chunk * rt.sb * tsz));
  TransBufs tb;
  TRY_RC(trans_bufs(ctx, p, g, rt.chunk * rt.sb, pl.tf, sc, &tb));
  const SpecIO io{g->nsel, nullptr, g->nsel, (int64_t)nq, g->qsel};
  for (int blk = 0; blk < pl.nblocks; ++blk) {
    const int p0 = blk * pl.Pb, Pbc = std::min(pl.Pb, P - p0);
    if (Pbc <= 0) break;
    Scratch bsc(st);  // released on the stream at the end of the block
    float2* psi0 = nullptr;
    if (pr.psi0) {
      psi0 = const_cast<float2*>(reinterpret_cast<const float2*>(pr.psi0)) + (size_t)p0 * nq;
    } else if (pr.alpha_mrad > 0.0) {
      tacaw_probe sub = pr;
      sub.n_probes = Pbc;
      sub.xy = pr.xy ? pr.xy + 2 * (size_t)p0 : nullptr;
      TRY_RC(build_probes(ctx, p, sub, bsc, &psi0));
    }
    float2 *psi_k, *Apsi, *Bpsi;
    CK(bsc.get(&psi_k, (size_t)Pbc * F * g->nsel));
    CK(bsc.get(&Apsi, (size_t)rt.chunk * Pbc * plane));
    CK(bsc.get(&Bpsi, (size_t)rt.chunk * Pbc * plane));
    const bool build_t = blk == 0 || !pl.keep_t;
    for (int64_t f0 = 0; f0 < F; f0 += rt.chunk) {
      const int nfc = (int)std::min<int64_t>(rt.chunk, F - f0);
      for (int s0 = 0; s0 < S; s0 += rt.sb) {
        const int sbc = std::min(rt.sb, S - s0);
        float2* tblk = pl.keep_t ? t + (size_t)f0 * S * tsz : t;
        if (build_t) {
          TRY_RC(potential_block(ctx, p, g, bn, A, f0, nfc, s0, sbc, Bp, Ap, st));
          NvtxRange r("transmission");
          TRY_RC(transmission_from(ctx, p, g, Ap, nullptr, nfc * sbc, tblk, sc, tb, pl.tf));
        }
        NvtxRange r("multislice");
        if (pl.keep_t)
          TRY_RC(slices(ctx, p, g, tblk, S, 0, nfc, s0, sbc, Pbc, psi0, F, f0, psi_k, true, sc, Apsi, Bpsi, pl.tf));
        else
          TRY_RC(slices(ctx, p, g, tblk, sbc, s0, nfc, s0, sbc, Pbc, psi0, F, f0, psi_k, true, sc, Apsi, Bpsi,
                        pl.tf));
      }
    }
    NvtxRange r("time_dft");
    float* out = d_S + (reduce == TACAW_REDUCE_NONE ? (size_t)p0 * F * nq : (size_t)p0 * F);
    TRY_RC(spectrum_impl(ctx, psi_k, (int64_t)Pbc * R, Fr, io, precision, reduce, out, bsc));
  }
  return TACAW_OK;
}

}  // namespace tacaw

extern "C" {

int tacaw_bin_slices(tacaw_ctx* ctx, const tacaw_params* params, const float* pos, int64_t n_atoms, int64_t nf,
                     int32_t* slice_out, void* stream) {
  if (!ctx) return TACAW_EINVAL;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  tacaw::NvtxRange nvtx("tacaw_bin_slices");
  TRY_RC(check_params(ctx, params));
  if (n_atoms < 0 || nf < 1) return set_err(ctx, TACAW_EINVAL, "n_atoms >= 0 and nf >= 1 required");
  if (n_atoms == 0) return TACAW_OK;
  if (!is_device_ptr(pos) || !is_device_ptr(slice_out)) return set_err(ctx, TACAW_EINVAL, "pos, slice_out must be device pointers");
  CK(cudaSetDevice(ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  Scratch sc(st);
  int* offs;
  CK(sc.get(&offs, (size_t)nf * (params->n_slices + 1)));
  CK(launch_bin(pos, n_atoms, nf, params->n_slices, params->cell[0], params->cell[1], params->cell[2], params->nx,
                params->ny, nullptr, nullptr, offs, slice_out, st));
  return TACAW_OK;
}

int tacaw_build_potential(tacaw_ctx* ctx, const tacaw_params* params, const float* pos, const int32_t* Z,
                          int64_t n_atoms, int64_t nf, float* V_out, void* stream) {
  if (!ctx) return TACAW_EINVAL;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  tacaw::NvtxRange nvtx("tacaw_build_potential");
  TRY_RC(check_params(ctx, params));
  const tacaw_params& p = *params;
  if (n_atoms < 0 || nf < 1) return set_err(ctx, TACAW_EINVAL, "n_atoms >= 0 and nf >= 1 required");
  TRY_RC(check_spread_band(ctx, params));
  if (ctx->ffZ.empty()) return set_err(ctx, TACAW_EINVAL, "no form-factor table loaded");
  if ((n_atoms > 0 && (!is_device_ptr(pos) || !is_device_ptr(Z))) || !is_device_ptr(V_out))
    return set_err(ctx, TACAW_EINVAL, "pos, Z and V_out must be device pointers");
  CK(cudaSetDevice(ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  GeoCache* g;
  TRY_RC(get_geo(ctx, p, &g));
  Scratch sc(st);
  int8_t* slots;
  TRY_RC(make_slots(ctx, Z, n_atoms, true, false, sc, &slots));
  const Geo geo{p.nx, p.ny, ctx->tw};
  const size_t plane = (size_t)p.ny * g->band.Wp;
  const int64_t chunk = chunk_frames(nf, p.n_slices * plane * 8 * (g->npair + 1), (size_t)1 << 30);
  return potential_chunks(ctx, p, g, pos, slots, n_atoms, nf, chunk, p.n_slices, sc,
                          [&](int64_t f0, int nfc, int, int, float2* Ap) {
    CK(launch_row_pot_out(geo, g->band, Ap, nfc * p.n_slices, 0, 0.f,
                          V_out + (size_t)f0 * p.n_slices * p.ny * p.nx, nullptr, (int)ctx->static_band, st));
    return TACAW_OK;
  });
}

int tacaw_transmission(tacaw_ctx* ctx, const tacaw_params* params, const float* V, int64_t nf, float* t_out,
                       void* stream) {
  if (!ctx) return TACAW_EINVAL;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  tacaw::NvtxRange nvtx("tacaw_transmission");
  TRY_RC(check_params(ctx, params));
  if (nf < 1) return set_err(ctx, TACAW_EINVAL, "nf >= 1 required");
  if (!is_device_ptr(V) || !is_device_ptr(t_out)) return set_err(ctx, TACAW_EINVAL, "V, t_out must be device pointers");
  CK(cudaSetDevice(ctx->device));
  GeoCache* g;
  TRY_RC(get_geo(ctx, *params, &g));
  Scratch sc((cudaStream_t)stream);
  const int64_t nfs = nf * params->n_slices;
  const int64_t step = std::min<int64_t>(nfs, 1024);
  TransBufs tb;
  TRY_RC(trans_bufs(ctx, *params, g, step, false, sc, &tb));
  for (int64_t i = 0; i < nfs; i += step) {
    const int n = (int)std::min(step, nfs - i);
    const size_t off = (size_t)i * params->ny * params->nx;
    TRY_RC(transmission_from(ctx, *params, g, nullptr, V + off, n, reinterpret_cast<float2*>(t_out) + off, sc, tb));
  }
  return TACAW_OK;
}

int tacaw_propagate(tacaw_ctx* ctx, const tacaw_params* params, const float* V, int64_t nf, const tacaw_probe* probe,
                    float* psi_k_out, void* stream) {
  if (!ctx) return TACAW_EINVAL;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  tacaw::NvtxRange nvtx("tacaw_propagate");
  TRY_RC(check_params(ctx, params));
  const tacaw_params& p = *params;
  tacaw_probe pr = probe ? *probe : default_probe();
  if (nf < 1 || pr.n_probes < 1) return set_err(ctx, TACAW_EINVAL, "nf >= 1 and n_probes >= 1 required");
  if (pr.alpha_mrad <= 0.0 && !pr.psi0 && pr.n_probes != 1)
    return set_err(ctx, TACAW_EINVAL, "a plane wave takes exactly one probe");
  if (pr.psi0 && !is_device_ptr(pr.psi0)) return set_err(ctx, TACAW_EINVAL, "probe psi0 must be a device pointer");
  if (!is_device_ptr(V) || !is_device_ptr(psi_k_out)) return set_err(ctx, TACAW_EINVAL, "V, psi_k_out must be device pointers");
  CK(cudaSetDevice(ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  GeoCache* g;
  TRY_RC(get_geo(ctx, p, &g));
  Scratch sc(st);
  const int P = pr.n_probes, S = p.n_slices;
  const size_t nq = (size_t)p.nx * p.ny, plane = (size_t)p.ny * g->band.Wp;
  float2* psi_k = reinterpret_cast<float2*>(psi_k_out);
  CK(cudaMemsetAsync(psi_k, 0, sizeof(float2) * nq * P * nf, st));
  float2* psi0 = nullptr;
  if (pr.psi0) psi0 = const_cast<float2*>(reinterpret_cast<const float2*>(pr.psi0));
  else if (pr.alpha_mrad > 0.0) TRY_RC(build_probes(ctx, p, pr, sc, &psi0));
  const size_t per_frame = (size_t)S * nq * 8 + (size_t)P * plane * 16;
  const int64_t chunk = chunk_frames(nf, per_frame, (size_t)2 << 30);
  float2 *t, *Apsi, *Bpsi;
  CK(sc.get(&t, (size_t)chunk * S * nq));
  CK(sc.get(&Apsi, (size_t)chunk * P * plane));
  CK(sc.get(&Bpsi, (size_t)chunk * P * plane));
  const bool tf = use_compact_t(p, P);
  TransBufs tb;
  TRY_RC(trans_bufs(ctx, p, g, chunk * S, tf, sc, &tb));
  for (int64_t f0 = 0; f0 < nf; f0 += chunk) {
    const int nfc = (int)std::min<int64_t>(chunk, nf - f0);
    TRY_RC(transmission_from(ctx, p, g, nullptr, V + (size_t)f0 * S * nq, nfc * S, t, sc, tb, tf));
    TRY_RC(slices(ctx, p, g, t, S, 0, nfc, 0, S, P, psi0, nf, f0, psi_k, false, sc, Apsi, Bpsi, tf));
  }
  return TACAW_OK;
}

int tacaw_spectrum(tacaw_ctx* ctx, const float* psi_k, int64_t P, int64_t F, int64_t nq, int32_t precision,
                   int32_t reduce, const int32_t* q_sel, int64_t n_sel, float* S_out, void* stream) {
  if (!ctx) return TACAW_EINVAL;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  tacaw::NvtxRange nvtx("tacaw_spectrum");
  if (P < 1 || F < 1 || nq < 1) return set_err(ctx, TACAW_EINVAL, "P, F, nq must be >= 1");
  if (!is_device_ptr(psi_k) || !is_device_ptr(S_out) || (q_sel && !is_device_ptr(q_sel)))
    return set_err(ctx, TACAW_EINVAL, "psi_k, S_out (and q_sel) must be device pointers");
  if (q_sel && (n_sel < 1 || n_sel > nq)) return set_err(ctx, TACAW_EINVAL, "n_sel must be in [1, nq]");
  CK(cudaSetDevice(ctx->device));
  Scratch sc((cudaStream_t)stream);
  const SpecIO io{nq, q_sel, q_sel ? n_sel : nq, nq, q_sel};
  return spectrum_impl(ctx, reinterpret_cast<const float2*>(psi_k), P, F, io, precision, reduce, S_out, sc);
}

int tacaw_run(tacaw_ctx* ctx, const tacaw_params* params, const float* pos, const int32_t* Z, int64_t n_atoms,
              int64_t n_frames, const tacaw_probe* probe, int32_t precision, int32_t reduce, float* S_out,
              void* stream) {
  if (!ctx) return TACAW_EINVAL;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  tacaw::NvtxRange nvtx("tacaw_run");
  tacaw_probe pr = probe ? *probe : default_probe();
  TRY_RC(check_run(ctx, params, pr, pos, Z, n_atoms, n_frames, precision, reduce, S_out, true));
  const tacaw_params& p = *params;
  CK(cudaSetDevice(ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  Scratch sc(st);
  const int64_t F = n_frames, A = n_atoms;
  const size_t nq = (size_t)p.nx * p.ny;
  const bool pos_dev = A > 0 && is_device_ptr(pos), z_dev = A > 0 && is_device_ptr(Z);
  const float* d_pos = pos;
  if (A > 0 && !pos_dev) {
    float* tmp;
    CK(sc.get(&tmp, (size_t)F * A * 3));
    ProfScope ps(ctx, "h2d_pos", st, (double)sizeof(float) * F * A * 3, 0);
    CK(cudaMemcpyAsync(tmp, pos, sizeof(float) * F * A * 3, cudaMemcpyHostToDevice, st));
    d_pos = tmp;
  }
  const bool out_dev = is_device_ptr(S_out);
  const size_t out_elems = reduce == TACAW_REDUCE_NONE ? (size_t)pr.n_probes * F * nq : (size_t)pr.n_probes * F;
  float* d_S = S_out;
  if (!out_dev) CK(sc.get(&d_S, out_elems));
  TRY_RC(run_impl(ctx, p, pr, d_pos, Z, z_dev, A, F, precision, reduce, d_S, st, 1));
  if (!out_dev) {
    {
      ProfScope ps(ctx, "d2h_S", st, (double)sizeof(float) * out_elems, 0);
      CK(copy_to_host(ctx, S_out, d_S, out_elems, st));
    }
    CK(cudaStreamSynchronize(st));
  } else if (!pos_dev && A > 0) {
    CK(cudaStreamSynchronize(st));  // the caller's host positions were read asynchronously
  }
  return TACAW_OK;
}

int tacaw_band_points(tacaw_ctx* ctx, const tacaw_params* params, int32_t* q_out, int64_t* n_out) {
  if (!ctx || !n_out) return TACAW_EINVAL;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  TRY_RC(check_params(ctx, params));
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_err(ctx, e, "cudaSetDevice");
  GeoCache* g;
  const int rc = get_geo(ctx, *params, &g);
  if (rc != TACAW_OK) return rc;
  *n_out = g->nsel;
  if (q_out) {
    e = cudaMemcpy(q_out, g->qsel, sizeof(int32_t) * g->nsel, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_err(ctx, e, "band points copy");
  }
  return TACAW_OK;
}

int tacaw_set_option(tacaw_ctx* ctx, const char* name, int64_t value) {
  if (!ctx || !name) return TACAW_EINVAL;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  if (std::strcmp(name, "max_chunk_frames") == 0) {
    if (value < 0) return set_err(ctx, TACAW_EINVAL, "max_chunk_frames must be >= 0");
    ctx->max_chunk_frames = value;
    return TACAW_OK;
  }
  if (std::strcmp(name, "min_wave_rows") == 0) {
    if (value < 0) return set_err(ctx, TACAW_EINVAL, "min_wave_rows must be >= 0");
    ctx->min_wave_rows = value;
    return TACAW_OK;
  }
  if (std::strcmp(name, "max_slice_block") == 0) {
    if (value < 0) return set_err(ctx, TACAW_EINVAL, "max_slice_block must be >= 0");
    ctx->max_slice_block = value;
    return TACAW_OK;
  }
  if (std::strcmp(name, "max_run_bytes") == 0) {
    if (value < 0) return set_err(ctx, TACAW_EINVAL, "max_run_bytes must be >= 0");
    ctx->max_run_bytes = value;
    return TACAW_OK;
  }
  if (std::strcmp(name, "serving_streams") == 0) {
    if (value < 1 || value > 64) return set_err(ctx, TACAW_EINVAL, "serving_streams must be in [1, 64]");
    if (ctx->serving) return set_err(ctx, TACAW_EINVAL, "serving_streams must be set before the first tacaw_submit");
    ctx->serving_streams = value;
    return TACAW_OK;
  }
  if (std::strcmp(name, "serving_small_work") == 0) {
    if (value < 0) return set_err(ctx, TACAW_EINVAL, "serving_small_work must be >= 0");
    ctx->serving_small_work = value;
    return TACAW_OK;
  }
  if (std::strcmp(name, "static_band") == 0) {
    if (value < 0 || value > 1) return set_err(ctx, TACAW_EINVAL, "static_band must be 0 or 1");
    ctx->static_band = value;
    return TACAW_OK;
  }
  if (std::strcmp(name, "host_copy") == 0) {
    if (value < 0 || value > 1) return set_err(ctx, TACAW_EINVAL, "host_copy must be 0 or 1");
    ctx->host_copy = value;
    return TACAW_OK;
  }
  if (std::strcmp(name, "max_coalesce") == 0) {
    if (value < 1 || value > 1024) return set_err(ctx, TACAW_EINVAL, "max_coalesce must be in [1, 1024]");
    ctx->max_coalesce = value;
    return TACAW_OK;
  }
  if (std::strcmp(name, "max_probe_block") == 0) {
    if (value < 0) return set_err(ctx, TACAW_EINVAL, "max_probe_block must be >= 0");
    ctx->max_probe_block = value;
    return TACAW_OK;
  }
  return set_err(ctx, TACAW_EINVAL, "unknown option '%s'", name);
}

int tacaw_check(tacaw_ctx* ctx) {
  if (!ctx) return TACAW_EINVAL;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  CK(cudaSetDevice(ctx->device));
  CK(cudaDeviceSynchronize());
  int st = 0;
  CK(cudaMemcpy(&st, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  if (st != 0) {
    CK(cudaMemset(ctx->d_status, 0, sizeof(int)));
    if (st & TACAW_STATUS_TIMEOUT)
      return set_err(ctx, TACAW_ETIMEOUT, "a kernel's bounded wait ran out (status %d); its results are invalid", st);
    return set_err(ctx, TACAW_EINVAL,
                   "an atom's Z was not in the form-factor table (Z on the device); the results of that run are "
                   "invalid");
  }
  return TACAW_OK;
}

int tacaw_profile_begin(tacaw_ctx* ctx) {
  if (!ctx) return TACAW_EINVAL;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  ctx->prof.recs.clear();
  ctx->prof.next = 0;
  ctx->prof.on = true;
  return TACAW_OK;
}

int tacaw_profile_select(tacaw_ctx* ctx, const char* names) {
  if (!ctx) return TACAW_EINVAL;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  if (ctx->prof.on) return set_err(ctx, TACAW_EINVAL, "tacaw_profile_select while a profile is being recorded");
  ctx->prof.select.clear();
  if (!names) return TACAW_OK;
  std::string cur;
  for (const char* c = names;; ++c) {
    if (*c == ',' || *c == 0) {
      if (!cur.empty()) ctx->prof.select.push_back(cur);
      cur.clear();
      if (*c == 0) break;
    } else if (*c != ' ') {
      cur.push_back(*c);
    }
  }
  return TACAW_OK;
}
int tacaw_profile_end(tacaw_ctx* ctx, char* names, double* ms, int64_t* launches, double* bytes, double* flops,
                      int32_t max_n, int32_t* n_out) {
  if (!ctx) return TACAW_EINVAL;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  ctx->prof.on = false;
  std::vector<std::string> order;
  std::map<std::string, std::tuple<double, int64_t, double, double>> acc;
  for (const ProfRec& r : ctx->prof.recs) {
    float t = 0.f;
    if (r.a) {
      CK(cudaEventSynchronize(r.b));
      CK(cudaEventElapsedTime(&t, r.a, r.b));
    }
    if (!acc.count(r.name)) order.push_back(r.name);
    auto& a = acc[r.name];
    std::get<0>(a) += t;
    std::get<1>(a) += 1;
    std::get<2>(a) += r.bytes;
    std::get<3>(a) += r.flops;
  }
  ctx->prof.recs.clear();
  ctx->prof.next = 0;
  const int n = (int)order.size();
  if (n_out) *n_out = n;
  for (int i = 0; i < n && i < max_n; ++i) {
    const auto& a = acc[order[i]];
    if (names) {
      std::strncpy(names + 32 * i, order[i].c_str(), 31);
      names[32 * i + 31] = 0;
    }
    if (ms) ms[i] = std::get<0>(a);
    if (launches) launches[i] = std::get<1>(a);
    if (bytes) bytes[i] = std::get<2>(a);
    if (flops) flops[i] = std::get<3>(a);
  }
  return TACAW_OK;
}

}  // extern "C"

namespace tacaw {

int spectrum_impl(tacaw_ctx* ctx, const float2* psi_k, int64_t P, int64_t F, const SpecIO& io, int32_t precision,
                  int32_t reduce, float* S_out, Scratch& sc) {
  if (reduce != TACAW_REDUCE_NONE && reduce != TACAW_REDUCE_DETECTOR) return set_err(ctx, TACAW_EINVAL, "bad reduce");
  if (precision < TACAW_DFT_FP32 || precision > TACAW_DFT_TF32) return set_err(ctx, TACAW_EINVAL, "bad precision");
  cudaStream_t st = sc.st;
  const int64_t nsel = io.nsel;
  const double pfq = (double)P * F * nsel;
  const bool det = reduce == TACAW_REDUCE_DETECTOR;
  if (!det && io.out_qsel && nsel < io.out_nq) CK(cudaMemsetAsync(S_out, 0, sizeof(float) * P * F * io.out_nq, st));
  if (precision == TACAW_DFT_FP32) {
    double2* mean;
    CK(sc.get(&mean, (size_t)P * nsel));
    {
      ProfScope ps(ctx, "mean_f64", st, pfq * 8 + (double)P * nsel * 16, pfq * 2);
      CK(launch_mean_f64(psi_k, P, F, io.in_nq, io.in_qsel, nsel, mean, st));
    }
    float2* r;
    CK(sc.get(&r, (size_t)P * F * nsel));
    {
      ProfScope ps(ctx, "residual_f32", st, pfq * 16, pfq * 2);
      CK(launch_residual_f32(psi_k, mean, P, F, io.in_nq, io.in_qsel, nsel, r, st));
    }
    float2* twF;
    TRY_RC(get_time_tw(ctx, F, &twF));
    // the detector sum reads a compact S [P][F][nsel]
    float* S = S_out;
    if (det) CK(sc.get(&S, (size_t)P * F * nsel));
    {
      ProfScope ps(ctx, "dft_fp32", st, pfq * 12, pfq * 8.0 * F);
      CK(launch_dft_fp32(r, twF, P, F, nsel, det ? nsel : io.out_nq, det ? nullptr : io.out_qsel, S, st));
    }
    if (det) {
      ProfScope ps(ctx, "detector_reduce", st, pfq * 4, pfq);
      CK(launch_detector_reduce(S, P, F, nsel, nullptr, nsel, S_out, st));
    }
    return TACAW_OK;
  }
  return spectrum_tc(ctx, psi_k, P, F, io, precision, reduce, S_out, sc);
}

}  // namespace tacaw
