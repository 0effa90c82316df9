// QQ^T driven by a precomputed sorted index map (Sec. 2.1, direct stiffness summation), for any
// element connectivity.
//
// Q maps global nodes to local copies, so (QQ^T u)_l is the sum of u over every local copy of
// l's global node.  The map lists the local ids of each global node that has more than one copy,
// grouped by global id, in four buckets by multiplicity (groups of 2, 4 and 8 copies at fixed
// width, groups of any other count as CSR segments), plus the single copies of Dirichlet nodes
// (zeroed when the mask is applied).  A global node is Dirichlet when any of its copies is
// flagged; the first id of a Dirichlet group is stored as ~id.  Within a group the copies are in
// ascending local id and are summed in that order, from the first; groups are ordered by their
// first copy, which keeps the first copies' reads close together in memory.
//
// The box-lattice meshes of this library default to QQ^T as three direction sweeps (ax.cu), which
// need no map; this path serves any numbering (se_gsmap_*) and, with SE_MESH_GS_MAP, every level
// of a mesh and of its preconditioners.  Each shared copy costs one 4-byte id read plus one value
// read and one value write: HBM-bound.
#include <algorithm>
#include <cstring>
#include <utility>

#include "se_internal.h"

namespace se {

constexpr int GSM_PAIRS = 4;  // pairs per thread (interleaved, so a warp's id loads coalesce)

static inline int64_t round4(int64_t n) { return (n + 3) / 4 * 4; }

// ------------------------------------------------------------------ host construction
struct GsMapHost {
  std::vector<int> b2, b4, b8, gen, goff, single;
};

static int gsmap_validate(int64_t L, const int64_t* gid) {
  SE_CHECK(L > 0 && L < ((int64_t)1 << 31), SE_EINVAL, "gsmap: L = %lld out of range (1 .. 2^31-1)",
           (long long)L);
  SE_CHECK(gid != nullptr, SE_EINVAL, "gsmap: null global id array");
  for (int64_t l = 0; l < L; ++l)
    SE_CHECK(gid[l] >= 0, SE_EINVAL, "gsmap: negative global id %lld at local point %lld",
             (long long)gid[l], (long long)l);
  return SE_OK;
}

// Groups the local ids by global id (ascending local id within a group) and fills the buckets.
static int gsmap_build_host(int64_t L, const int64_t* gid, const uint8_t* dir, GsMapHost& h) {
  SE_TRY(gsmap_validate(L, gid));
  int64_t gmax = 0;
  for (int64_t l = 0; l < L; ++l) gmax = std::max(gmax, gid[l]);
  std::vector<int> order((size_t)L);        // local ids grouped by global id
  std::vector<int64_t> gstart, gsize;       // groups in global id order
  if (gmax < 2 * L + 1024) {                // compact numbering: counting sort
    std::vector<int64_t> cnt((size_t)gmax + 2, 0);  // cnt[g + 1]: copies of g, then prefix sums
    for (int64_t l = 0; l < L; ++l) ++cnt[(size_t)gid[l] + 1];
    for (int64_t g = 0; g <= gmax; ++g) cnt[(size_t)g + 1] += cnt[(size_t)g];
    for (int64_t g = 0; g <= gmax; ++g)
      if (cnt[(size_t)g + 1] > cnt[(size_t)g]) {
        gstart.push_back(cnt[(size_t)g]);
        gsize.push_back(cnt[(size_t)g + 1] - cnt[(size_t)g]);
      }
    for (int64_t l = 0; l < L; ++l) order[(size_t)cnt[(size_t)gid[l]]++] = (int)l;
  } else {                                   // sparse labels: sort (global id, local id) pairs
    std::vector<std::pair<int64_t, int>> v((size_t)L);
    for (int64_t l = 0; l < L; ++l) v[(size_t)l] = {gid[l], (int)l};
    std::sort(v.begin(), v.end());
    for (int64_t i = 0; i < L; ++i) {
      order[(size_t)i] = v[(size_t)i].second;
      if (i == 0 || v[(size_t)i].first != v[(size_t)i - 1].first) {
        gstart.push_back(i);
        gsize.push_back(0);
      }
      ++gsize.back();
    }
  }
  // emit the groups in the order of their first (smallest) local id
  std::vector<int> first_of((size_t)L, -1);  // group index whose first copy is local point l
  for (size_t g = 0; g < gstart.size(); ++g) first_of[(size_t)order[(size_t)gstart[g]]] = (int)g;
  h.goff.push_back(0);
  for (int64_t l = 0; l < L; ++l) {
    const int g = first_of[(size_t)l];
    if (g < 0) continue;
    const int* ids = order.data() + gstart[(size_t)g];
    const int64_t m = gsize[(size_t)g];
    bool masked = false;
    if (dir)
      for (int64_t c = 0; c < m; ++c) masked |= dir[ids[c]] != 0;
    if (m == 1) {
      if (masked) h.single.push_back(ids[0]);
      continue;
    }
    std::vector<int>& dst = m == 2 ? h.b2 : m == 4 ? h.b4 : m == 8 ? h.b8 : h.gen;
    dst.push_back(masked ? ~ids[0] : ids[0]);
    for (int64_t c = 1; c < m; ++c) dst.push_back(ids[c]);
    if (m != 2 && m != 4 && m != 8) h.goff.push_back((int)h.gen.size());
  }
  return SE_OK;
}

static void gsmap_counts(const GsMapHost& h, int64_t counts[5]) {
  counts[0] = (int64_t)h.b2.size() / 2;
  counts[1] = (int64_t)h.b4.size() / 4;
  counts[2] = (int64_t)h.b8.size() / 8;
  counts[3] = (int64_t)h.goff.size() - 1;
  counts[4] = (int64_t)h.single.size();
}

// Uploads the buckets into lv.gsm_* (each bucket at a multiple of 4 ints, so the vector loads of
// the pair, quad and octet ids are aligned).
static int gsmap_upload(const GsMapHost& h, Level& lv, Allocs& allocs, cudaStream_t s) {
  int64_t n[5];
  gsmap_counts(h, n);
  const std::vector<int>* seg[5] = {&h.b2, &h.b4, &h.b8, &h.gen, &h.single};
  int64_t total = 0;
  for (int b = 0; b < 5; ++b) {
    lv.gsm_seg[b] = total;
    total += round4((int64_t)seg[b]->size());
  }
  std::vector<int> flat((size_t)total + 4, 0);
  for (int b = 0; b < 5; ++b)
    if (!seg[b]->empty())
      std::memcpy(flat.data() + lv.gsm_seg[b], seg[b]->data(), seg[b]->size() * sizeof(int));
  SE_TRY(dmalloc(allocs, &lv.gsm_ids, flat.size()));
  SE_TRY(dmalloc(allocs, &lv.gsm_goff, h.goff.size()));
  SE_CUDA(cudaMemcpyAsync(lv.gsm_ids, flat.data(), flat.size() * sizeof(int), cudaMemcpyHostToDevice, s));
  SE_CUDA(cudaMemcpyAsync(lv.gsm_goff, h.goff.data(), h.goff.size() * sizeof(int),
                          cudaMemcpyHostToDevice, s));
  SE_CUDA(cudaStreamSynchronize(s));  // the host buffers go out of scope
  for (int b = 0; b < 5; ++b) lv.gsm_n[b] = n[b];
  lv.gsm_entries = 2 * n[0] + 4 * n[1] + 8 * n[2] + (int64_t)h.gen.size();
  return SE_OK;
}

// The map of a box-lattice level (SE_MESH_GS_MAP): global lattice ids and Dirichlet flags from
// the device, grouped on the host.
int build_level_gsmap(Level& lv, Allocs& allocs, cudaStream_t s) {
  int* l2g = nullptr;
  SE_TRY(dmalloc_transient(reinterpret_cast<void**>(&l2g), (size_t)lv.L * sizeof(int), s));
  int st = local_to_global(lv, l2g, s);
  std::vector<int> g32((size_t)lv.L);
  std::vector<uint8_t> pf((size_t)lv.L);
  if (st == SE_OK &&
      (cudaMemcpyAsync(g32.data(), l2g, (size_t)lv.L * sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
       cudaMemcpyAsync(pf.data(), lv.pflag, (size_t)lv.L, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
       cudaStreamSynchronize(s) != cudaSuccess)) {
    set_error("gsmap: %s", cudaGetErrorString(cudaGetLastError()));
    st = SE_ECUDA;
  }
  cudaFreeAsync(l2g, s);
  if (st != SE_OK) return st;
  std::vector<int64_t> gid(g32.begin(), g32.end());
  std::vector<uint8_t> dir((size_t)lv.L);
  for (int64_t l = 0; l < lv.L; ++l) dir[(size_t)l] = (pf[(size_t)l] & PF_FREE) ? 0 : 1;
  GsMapHost h;
  SE_TRY(gsmap_build_host(lv.L, gid.data(), dir.data(), h));
  return gsmap_upload(h, lv, allocs, s);
}

int build_gsmap_from_gid(Level& lv, const int64_t* gid, const uint8_t* dirichlet, Allocs& allocs,
                         cudaStream_t s) {
  SE_TRY(gsmap_validate(lv.L, gid));
  GsMapHost h;
  SE_TRY(gsmap_build_host(lv.L, gid, dirichlet, h));
  return gsmap_upload(h, lv, allocs, s);
}

// ------------------------------------------------------------------ device
template <typename T, int M>
__device__ __forceinline__ void gsm_group(const int* __restrict__ ids, T* __restrict__ u, bool mask) {
  int id[M];
#pragma unroll
  for (int q = 0; q < M; q += 4) {
    const int4 v = *reinterpret_cast<const int4*>(ids + q);
    id[q] = v.x;
    id[q + 1] = v.y;
    id[q + 2] = v.z;
    id[q + 3] = v.w;
  }
  const bool masked = id[0] < 0;
  if (masked) id[0] = ~id[0];
  T val[M];
#pragma unroll
  for (int c = 0; c < M; ++c) val[c] = u[id[c]];
  T sum = val[0];
#pragma unroll
  for (int c = 1; c < M; ++c) sum += val[c];
  if (masked && mask) sum = T(0);
#pragma unroll
  for (int c = 0; c < M; ++c) u[id[c]] = sum;
}

// Thread ranges, in order: pairs (GSM_PAIRS per thread), quads, octets, other groups, masked
// single copies.
template <typename T>
__global__ void __launch_bounds__(256) gsmap_kernel(int64_t n2, int64_t n4, int64_t n8, int64_t ng,
                                                    int64_t n1, const int* __restrict__ ids2,
                                                    const int* __restrict__ ids4,
                                                    const int* __restrict__ ids8,
                                                    const int* __restrict__ idsg,
                                                    const int* __restrict__ goff,
                                                    const int* __restrict__ ids1, T* __restrict__ u,
                                                    bool mask) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t T2 = (n2 + GSM_PAIRS - 1) / GSM_PAIRS;
  if (t < T2) {
    int a[GSM_PAIRS], b[GSM_PAIRS];
    bool on[GSM_PAIRS], ms[GSM_PAIRS];
#pragma unroll
    for (int k = 0; k < GSM_PAIRS; ++k) {
      const int64_t g = t + k * T2;
      on[k] = g < n2;
      const int2 q = on[k] ? *reinterpret_cast<const int2*>(ids2 + 2 * g) : make_int2(0, 0);
      ms[k] = q.x < 0;
      a[k] = ms[k] ? ~q.x : q.x;
      b[k] = q.y;
    }
    T va[GSM_PAIRS], vb[GSM_PAIRS];
#pragma unroll
    for (int k = 0; k < GSM_PAIRS; ++k) {
      va[k] = on[k] ? u[a[k]] : T(0);
      vb[k] = on[k] ? u[b[k]] : T(0);
    }
#pragma unroll
    for (int k = 0; k < GSM_PAIRS; ++k) {
      if (!on[k]) continue;
      const T sum = (ms[k] && mask) ? T(0) : va[k] + vb[k];
      u[a[k]] = sum;
      u[b[k]] = sum;
    }
    return;
  }
  t -= T2;
  if (t < n4) {
    gsm_group<T, 4>(ids4 + 4 * t, u, mask);
    return;
  }
  t -= n4;
  if (t < n8) {
    gsm_group<T, 8>(ids8 + 8 * t, u, mask);
    return;
  }
  t -= n8;
  if (t < ng) {
    const int s0 = goff[t], s1 = goff[t + 1];
    int first = idsg[s0];
    const bool masked = first < 0;
    if (masked) first = ~first;
    T sum = u[first];
    for (int c = s0 + 1; c < s1; ++c) sum += u[idsg[c]];
    if (masked && mask) sum = T(0);
    u[first] = sum;
    for (int c = s0 + 1; c < s1; ++c) u[idsg[c]] = sum;
    return;
  }
  t -= ng;
  if (t < n1 && mask) u[ids1[t]] = T(0);
}

template <class T>
int gsmap_apply(const Level& lv, T* u, bool mask, cudaStream_t s) {
  const int64_t* n = lv.gsm_n;
  const int64_t threads = (n[0] + GSM_PAIRS - 1) / GSM_PAIRS + n[1] + n[2] + n[3] + n[4];
  if (threads == 0) return SE_OK;
  const double ent = (double)lv.gsm_entries;
  ProfScope prof(SE_K_GS, s, ent, ent * (2.0 * sizeof(T) + 4.0) + (mask ? n[4] * (4.0 + sizeof(T)) : 0.0),
                 ent, prof_variant<T>(lv.p));
  const int* I = lv.gsm_ids;
  gsmap_kernel<T><<<grid_for(threads, 256), 256, 0, s>>>(
      n[0], n[1], n[2], n[3], n[4], I + lv.gsm_seg[0], I + lv.gsm_seg[1], I + lv.gsm_seg[2],
      I + lv.gsm_seg[3], lv.gsm_goff, I + lv.gsm_seg[4], u, mask);
  SE_LAUNCH_CHECK();
  return SE_OK;
}

template int gsmap_apply<double>(const Level&, double*, bool, cudaStream_t);
template int gsmap_apply<float>(const Level&, float*, bool, cudaStream_t);

}  // namespace se

using namespace se;

struct se_gsmap_s {
  se::Allocs allocs;
  se::Level lv;
  cudaStream_t stream = nullptr;
};

extern "C" {

int se_gsmap_count(int64_t L, const int64_t* gid, const uint8_t* dirichlet, int64_t* counts) {
  SE_CHECK(counts != nullptr, SE_EINVAL, "se_gsmap_count: null counts");
  GsMapHost h;
  SE_TRY(gsmap_build_host(L, gid, dirichlet, h));
  gsmap_counts(h, counts);
  return SE_OK;
}

int se_gsmap_create(int64_t L, const int64_t* gid, const uint8_t* dirichlet, se_gsmap_t* out) {
  SE_CHECK(out != nullptr, SE_EINVAL, "se_gsmap_create: null output handle");
  *out = nullptr;
  GsMapHost h;
  SE_TRY(gsmap_build_host(L, gid, dirichlet, h));  // validates before any device work
  se_gsmap_s* g = new (std::nothrow) se_gsmap_s();
  SE_CHECK(g != nullptr, SE_ENOMEM, "se_gsmap_create: out of host memory");
  // a blocking stream, as for meshes: work the caller enqueues with stream == NULL is ordered with
  // the legacy default stream
  if (cudaStreamCreateWithFlags(&g->stream, cudaStreamDefault) != cudaSuccess) {
    delete g;
    set_error("se_gsmap_create: stream creation failed");
    return SE_ECUDA;
  }
  g->allocs.stream = g->stream;
  g->lv.L = L;
  g->lv.p = 0;
  const int st = gsmap_upload(h, g->lv, g->allocs, g->stream);
  if (st != SE_OK) {
    se_gsmap_destroy(g);
    return st;
  }
  *out = g;
  return SE_OK;
}

int se_gsmap_apply(se_gsmap_t g, double* u, int mask, void* stream) {
  SE_CHECK(g && u, SE_EINVAL, "se_gsmap_apply: null argument");
  return gsmap_apply<double>(g->lv, u, mask != 0, as_stream(stream, g->stream));
}

int se_gsmap_apply_f32(se_gsmap_t g, float* u, int mask, void* stream) {
  SE_CHECK(g && u, SE_EINVAL, "se_gsmap_apply_f32: null argument");
  return gsmap_apply<float>(g->lv, u, mask != 0, as_stream(stream, g->stream));
}

int se_gsmap_info(se_gsmap_t g, int64_t* counts) {
  SE_CHECK(g && counts, SE_EINVAL, "se_gsmap_info: null argument");
  for (int b = 0; b < 5; ++b) counts[b] = g->lv.gsm_n[b];
  return SE_OK;
}

int se_gsmap_destroy(se_gsmap_t g) {
  if (!g) return SE_OK;
  if (g->stream) cudaStreamSynchronize(g->stream);
  g->allocs.release();
  if (g->stream) {
    cudaStreamSynchronize(g->stream);
    cudaStreamDestroy(g->stream);
  }
  delete g;
  return SE_OK;
}

}  // extern "C"
