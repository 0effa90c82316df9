// Errors, allocations, 1D GLL basis, SplitMix64, reduction scratch and kernel profiling.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <mutex>

#include "se_internal.h"

namespace se {

static thread_local std::string g_last_error;

void set_error(const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
}

void Allocs::release() {
  for (void* p : ptrs) cudaFreeAsync(p, stream);
  ptrs.clear();
  bytes = 0;
}

// Self-test of the allocation failure paths (se_selftest_fail_alloc): while the countdown is
// positive every device allocation decrements it, and the one that brings it to zero fails with
// SE_ENOMEM before any CUDA call.
static std::atomic<int> g_fail_alloc_countdown{0};

static bool injected_alloc_failure() {
  int c = g_fail_alloc_countdown.load();
  while (c > 0 && !g_fail_alloc_countdown.compare_exchange_weak(c, c - 1)) {
  }
  return c == 1;
}

int dmalloc_transient(void** p, size_t bytes, cudaStream_t s) {
  if (injected_alloc_failure()) {
    *p = nullptr;
    set_error("device allocation of %zu bytes failed: injected by se_selftest_fail_alloc", bytes);
    return SE_ENOMEM;
  }
  cudaError_t e = cudaMallocAsync(p, bytes, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
    if (*p) cudaFreeAsync(*p, s);
    *p = nullptr;
    return SE_ENOMEM;
  }
  return SE_OK;
}

int dmalloc_bytes(Allocs& a, void** p, size_t bytes) {
  *p = nullptr;
  SE_TRY(dmalloc_transient(p, bytes, a.stream));
  a.ptrs.push_back(*p);
  a.bytes += bytes;
  return SE_OK;
}

void dfree(Allocs& a, void* p, size_t bytes) {
  auto it = std::find(a.ptrs.begin(), a.ptrs.end(), p);
  if (it == a.ptrs.end()) return;
  a.ptrs.erase(it);
  a.bytes -= bytes;
  cudaFreeAsync(p, a.stream);
}

int h2d(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  SE_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s));
  SE_CUDA(cudaStreamSynchronize(s));
  return SE_OK;
}

int dzero(void* p, size_t bytes, cudaStream_t s) {
  SE_CUDA(cudaMemsetAsync(p, 0, bytes, s));
  SE_CUDA(cudaStreamSynchronize(s));
  return SE_OK;
}

static std::mutex g_pin_mu;
static std::vector<double*> g_pin_free;

int pinned_scalars(double** out) {
  {
    std::lock_guard<std::mutex> g(g_pin_mu);
    if (!g_pin_free.empty()) {
      *out = g_pin_free.back();
      g_pin_free.pop_back();
      return SE_OK;
    }
  }
  SE_CUDA(cudaMallocHost(out, SCAL_SLOTS * sizeof(double)));
  return SE_OK;
}

void pinned_release(double* p) {
  if (!p) return;
  std::lock_guard<std::mutex> g(g_pin_mu);
  g_pin_free.push_back(p);
}

// ------------------------------------------------------------------ GLL basis (Sec. 2.1)
// Legendre P_n and its first two derivatives by the three-term recurrences
// P_{k+1} = ((2k+1) x P_k - k P_{k-1})/(k+1), P'_{k+1} = P'_{k-1} + (2k+1) P_k (and likewise
// for P'').
static void legendre3(int n, double x, double* P, double* dP, double* d2P) {
  double p0 = 1.0, p1 = x, d0 = 0.0, d1 = 1.0, s0 = 0.0, s1 = 0.0;
  if (n == 0) {
    *P = 1.0; *dP = 0.0; *d2P = 0.0;
    return;
  }
  for (int k = 1; k < n; ++k) {
    double p2 = ((2 * k + 1) * x * p1 - k * p0) / (k + 1);
    double d2 = d0 + (2 * k + 1) * p1;
    double s2 = s0 + (2 * k + 1) * d1;
    p0 = p1; p1 = p2; d0 = d1; d1 = d2; s0 = s1; s1 = s2;
  }
  *P = p1; *dP = d1; *d2P = s1;
}

void gll_basis(int p, Basis1D* b) {
  const int N = p + 1;
  b->p = p;
  b->xi[0] = -1.0;
  b->xi[p] = 1.0;
  // interior nodes: roots of P_p', Newton from the Chebyshev-Gauss-Lobatto points
  for (int j = 1; j < p; ++j) {
    double x = -std::cos(M_PI * j / p);
    for (int it = 0; it < 100; ++it) {
      double P, dP, d2P;
      legendre3(p, x, &P, &dP, &d2P);
      double dx = dP / d2P;
      x -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    b->xi[j] = x;
  }
  if (p % 2 == 0) b->xi[p / 2] = 0.0;
  double Pv[SE_MAX_ORDER + 1];
  for (int j = 0; j <= p; ++j) {
    double P, dP, d2P;
    legendre3(p, b->xi[j], &P, &dP, &d2P);
    Pv[j] = P;
    b->w[j] = 2.0 / (p * (p + 1) * P * P);
  }
  // closed-form GLL derivative matrix: D_ij = P_p(xi_i) / (P_p(xi_j) (xi_i - xi_j)), i != j;
  // D_00 = -p(p+1)/4, D_pp = p(p+1)/4, other diagonal entries 0.
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j) {
      double v;
      if (i != j) v = Pv[i] / (Pv[j] * (b->xi[i] - b->xi[j]));
      else if (i == 0) v = -0.25 * p * (p + 1);
      else if (i == p) v = 0.25 * p * (p + 1);
      else v = 0.0;
      b->D[i * N + j] = v;
    }
}

void interp_matrix(int pf, int pc, double* J) {
  Basis1D f, c;
  gll_basis(pf, &f);
  gll_basis(pc, &c);
  const int Nf = pf + 1, Nc = pc + 1;
  for (int i = 0; i < Nf; ++i)
    for (int j = 0; j < Nc; ++j) {
      double v = 1.0;
      for (int m = 0; m < Nc; ++m)
        if (m != j) v *= (f.xi[i] - c.xi[m]) / (c.xi[j] - c.xi[m]);
      J[i * Nc + j] = v;
    }
}

// ------------------------------------------------------------------ SplitMix64
uint64_t splitmix64(uint64_t seed, uint64_t c) { return splitmix64_hd(seed, c); }

double uniform01(uint64_t seed, uint64_t c) {
  return (double)(splitmix64(seed, c) >> 11) * (1.0 / 9007199254740992.0);
}

int scratch_alloc(Allocs& a, Scratch* s) {
  SE_TRY(dmalloc(a, &s->partial, (size_t)RED_MAX_BLOCKS * 4));
  SE_TRY(dmalloc(a, &s->counter, 1));
  SE_TRY(dmalloc(a, &s->scal, SCAL_SLOTS));
  SE_TRY(dzero(s->counter, sizeof(unsigned), a.stream));
  SE_TRY(dzero(s->scal, SCAL_SLOTS * sizeof(double), a.stream));
  SE_TRY(pinned_scalars(&s->hscal));
  return SE_OK;
}

// ------------------------------------------------------------------ launch tiles
static std::mutex g_tile_mu;
static TileCfg g_tiles[SE_MAX_ORDER + 1][2];

TileCfg tile_get(int p, bool fp32) {
  if (p < 0 || p > SE_MAX_ORDER) return TileCfg();
  std::lock_guard<std::mutex> g(g_tile_mu);
  return g_tiles[p][fp32 ? 1 : 0];
}

void tile_set(int p, bool fp32, const TileCfg& c) {
  if (p < 0 || p > SE_MAX_ORDER) return;
  std::lock_guard<std::mutex> g(g_tile_mu);
  g_tiles[p][fp32 ? 1 : 0] = c;
}

// ------------------------------------------------------------------ profiling
struct ProfEntry {
  int kind, variant;
  cudaEvent_t a, b;
  double units, bytes, flops;
};
struct ProfTotals {
  double ms = 0, units = 0, bytes = 0, flops = 0;
  int64_t launches = 0;
};
static std::mutex g_prof_mu;
static bool g_prof_on = false;
static std::vector<ProfEntry> g_prof_pending;
static std::vector<cudaEvent_t> g_prof_free;
static ProfTotals g_prof[SE_K_COUNT][PROF_VARIANTS];

static cudaEvent_t prof_event() {
  if (!g_prof_free.empty()) {
    cudaEvent_t e = g_prof_free.back();
    g_prof_free.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

static void prof_drain_locked() {
  for (auto& p : g_prof_pending) {
    cudaEventSynchronize(p.b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, p.a, p.b);
    auto& t = g_prof[p.kind][p.variant];
    t.ms += ms;
    t.launches += 1;
    t.units += p.units;
    t.bytes += p.bytes;
    t.flops += p.flops;
    g_prof_free.push_back(p.a);
    g_prof_free.push_back(p.b);
  }
  g_prof_pending.clear();
}

ProfScope::ProfScope(int kind_, cudaStream_t s_, double units_, double bytes_, double flops_,
                     int variant_)
    : kind(kind_), s(s_), units(units_), bytes(bytes_), flops(flops_),
      variant(variant_ >= 0 && variant_ < PROF_VARIANTS ? variant_ : 0), on(false) {
  std::lock_guard<std::mutex> g(g_prof_mu);
  if (!g_prof_on) return;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &cs);
  if (cs != cudaStreamCaptureStatusNone) return;  // no events inside a graph capture
  on = true;
  a = prof_event();
  b = prof_event();
  cudaEventRecord(a, s);
}

ProfScope::~ProfScope() {
  if (!on) return;
  std::lock_guard<std::mutex> g(g_prof_mu);
  cudaEventRecord(b, s);
  g_prof_pending.push_back({kind, variant, a, b, units, bytes, flops});
  if (g_prof_pending.size() > 4096) prof_drain_locked();
}

}  // namespace se

extern "C" {

const char* se_last_error(void) { return se::g_last_error.c_str(); }

int se_version(void) { return 1; }

int se_prof_enable(int on) {
  std::lock_guard<std::mutex> g(se::g_prof_mu);
  se::g_prof_on = on != 0;
  return SE_OK;
}

int se_prof_reset(void) {
  std::lock_guard<std::mutex> g(se::g_prof_mu);
  se::prof_drain_locked();
  for (auto& row : se::g_prof)
    for (auto& t : row) t = se::ProfTotals();
  return SE_OK;
}

int se_prof_query(int kind, double* ms_total, int64_t* launches, double* units, double* bytes,
                  double* flops) {
  return se_prof_query_variant(kind, -1, ms_total, launches, units, bytes, flops);
}

int se_prof_query_variant(int kind, int variant, double* ms_total, int64_t* launches,
                          double* units, double* bytes, double* flops) {
  SE_CHECK(kind >= 0 && kind < SE_K_COUNT, SE_EINVAL, "se_prof_query: bad kind %d", kind);
  SE_CHECK(variant >= -1 && variant < se::PROF_VARIANTS, SE_EINVAL, "se_prof_query: bad variant %d",
           variant);
  std::lock_guard<std::mutex> g(se::g_prof_mu);
  se::prof_drain_locked();
  se::ProfTotals t;
  for (int v = 0; v < se::PROF_VARIANTS; ++v) {
    if (variant >= 0 && v != variant) continue;
    const auto& x = se::g_prof[kind][v];
    t.ms += x.ms;
    t.launches += x.launches;
    t.units += x.units;
    t.bytes += x.bytes;
    t.flops += x.flops;
  }
  if (ms_total) *ms_total = t.ms;
  if (launches) *launches = t.launches;
  if (units) *units = t.units;
  if (bytes) *bytes = t.bytes;
  if (flops) *flops = t.flops;
  return SE_OK;
}

}  // extern "C"

extern "C" int se_selftest_fail_alloc(int n) {
  SE_CHECK(n >= 0, SE_EINVAL, "se_selftest_fail_alloc: n = %d < 0", n);
  se::g_fail_alloc_countdown.store(n);
  return SE_OK;
}
