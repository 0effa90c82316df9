// Mesh and level construction (Sec. 2.1): vertex lattice, isoparametric geometry, QQ^T index
// map, Dirichlet mask, multiplicities, element neighbours, Jacobi diagonal.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "pmg_internal.h"

namespace se {

// ------------------------------------------------------------------ geometry kernel
// One block per element, N*N threads (i, j), loop over k.  Node positions: trilinear map of the
// 8 lattice vertices to the GLL points, then x_c += amp sin(2 pi x) sin(2 pi y) sin(2 pi z).
// Geometric factors G_ab = w_i w_j w_k det(J) grad r_a . grad r_b = w adj(J) adj(J)^T / det(J).
__global__ void geometry_kernel(int N, int nx, int ny, const double* __restrict__ verts,
                                const double* __restrict__ xi, const double* __restrict__ wq,
                                const double* __restrict__ D, double amp, int64_t L,
                                double* __restrict__ X, double* __restrict__ G,
                                double* __restrict__ B) {
  extern __shared__ double smem[];
  const int N3 = N * N * N;
  double* sx = smem;            // [3][N3]
  double* sD = smem + 3 * N3;   // [N*N]
  const int e = blockIdx.x;
  const int ex = e % nx, ey = (e / nx) % ny, ez = e / (nx * ny);
  const int i = threadIdx.x % N, j = threadIdx.x / N;
  for (int t = threadIdx.x; t < N * N; t += blockDim.x) sD[t] = D[t];
  double cv[2][2][2][3];
  for (int dz = 0; dz < 2; ++dz)
    for (int dy = 0; dy < 2; ++dy)
      for (int dx = 0; dx < 2; ++dx) {
        int64_t v = (ex + dx) + (int64_t)(nx + 1) * ((ey + dy) + (int64_t)(ny + 1) * (ez + dz));
        for (int c = 0; c < 3; ++c) cv[dz][dy][dx][c] = verts[3 * v + c];
      }
  const double r = xi[i], s = xi[j];
  const double fr[2] = {0.5 * (1.0 - r), 0.5 * (1.0 + r)};
  const double fs[2] = {0.5 * (1.0 - s), 0.5 * (1.0 + s)};
  for (int k = 0; k < N; ++k) {
    const double t = xi[k];
    const double ft[2] = {0.5 * (1.0 - t), 0.5 * (1.0 + t)};
    double x[3] = {0.0, 0.0, 0.0};
    for (int dz = 0; dz < 2; ++dz)
      for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx) {
          const double wgt = ft[dz] * fs[dy] * fr[dx];
          for (int c = 0; c < 3; ++c) x[c] += wgt * cv[dz][dy][dx][c];
        }
    const double sm = sinpi(2.0 * x[0]) * sinpi(2.0 * x[1]) * sinpi(2.0 * x[2]);
    const int pt = i + N * (j + N * k);
    const int64_t gidx = (int64_t)e * N3 + pt;
    for (int c = 0; c < 3; ++c) {
      const double xc = x[c] + amp * sm;
      sx[c * N3 + pt] = xc;
      X[c * L + gidx] = xc;
    }
  }
  __syncthreads();
  for (int k = 0; k < N; ++k) {
    double Jm[3][3];  // Jm[c][a] = dx_c / dr_a
    for (int c = 0; c < 3; ++c) {
      const double* xc = sx + c * N3;
      double dr = 0.0, ds = 0.0, dt = 0.0;
      for (int l = 0; l < N; ++l) {
        dr += sD[i * N + l] * xc[l + N * (j + N * k)];
        ds += sD[j * N + l] * xc[i + N * (l + N * k)];
        dt += sD[k * N + l] * xc[i + N * (j + N * l)];
      }
      Jm[c][0] = dr; Jm[c][1] = ds; Jm[c][2] = dt;
    }
    // adj[a][c] = cofactor(Jm)[c][a]
    double adj[3][3];
    adj[0][0] = Jm[1][1] * Jm[2][2] - Jm[1][2] * Jm[2][1];
    adj[0][1] = Jm[0][2] * Jm[2][1] - Jm[0][1] * Jm[2][2];
    adj[0][2] = Jm[0][1] * Jm[1][2] - Jm[0][2] * Jm[1][1];
    adj[1][0] = Jm[1][2] * Jm[2][0] - Jm[1][0] * Jm[2][2];
    adj[1][1] = Jm[0][0] * Jm[2][2] - Jm[0][2] * Jm[2][0];
    adj[1][2] = Jm[0][2] * Jm[1][0] - Jm[0][0] * Jm[1][2];
    adj[2][0] = Jm[1][0] * Jm[2][1] - Jm[1][1] * Jm[2][0];
    adj[2][1] = Jm[0][1] * Jm[2][0] - Jm[0][0] * Jm[2][1];
    adj[2][2] = Jm[0][0] * Jm[1][1] - Jm[0][1] * Jm[1][0];
    const double det = Jm[0][0] * adj[0][0] + Jm[0][1] * adj[1][0] + Jm[0][2] * adj[2][0];
    const double wv = wq[i] * wq[j] * wq[k];
    const int64_t gidx = (int64_t)e * N3 + i + N * (j + N * k);
    const int ab[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
    const double sc = wv / det;
    for (int q = 0; q < 6; ++q) {
      const int a = ab[q][0], b = ab[q][1];
      G[q * L + gidx] = sc * (adj[a][0] * adj[b][0] + adj[a][1] * adj[b][1] + adj[a][2] * adj[b][2]);
    }
    B[gidx] = wv * det;
  }
}

// Per-point multiplicity, free bit and (optionally) global id.
__global__ void pointflag_kernel(int N, int nx, int ny, int nz, int64_t L, int bcmask,
                                 uint8_t* __restrict__ pflag, int* __restrict__ l2g) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= L) return;
  const int N3 = N * N * N, p = N - 1;
  const int64_t e = idx / N3;
  const int pt = (int)(idx - e * N3);
  const int i = pt % N, j = (pt / N) % N, k = pt / (N * N);
  const int ex = (int)(e % nx), ey = (int)((e / nx) % ny), ez = (int)(e / ((int64_t)nx * ny));
  const int I = ex * p + i, J = ey * p + j, K = ez * p + k;
  const int NX = nx * p + 1, NY = ny * p + 1, NZ = nz * p + 1;
  int mult = 1;
  if ((i == 0 && ex > 0) || (i == p && ex < nx - 1)) mult *= 2;
  if ((j == 0 && ey > 0) || (j == p && ey < ny - 1)) mult *= 2;
  if ((k == 0 && ez > 0) || (k == p && ez < nz - 1)) mult *= 2;
  bool fr = true;
  if ((bcmask & 1) && I == 0) fr = false;
  if ((bcmask & 2) && I == NX - 1) fr = false;
  if ((bcmask & 4) && J == 0) fr = false;
  if ((bcmask & 8) && J == NY - 1) fr = false;
  if ((bcmask & 16) && K == 0) fr = false;
  if ((bcmask & 32) && K == NZ - 1) fr = false;
  pflag[idx] = (uint8_t)(mult | (fr ? PF_FREE : 0));
  if (l2g) l2g[idx] = (int)(I + (int64_t)NX * (J + (int64_t)NY * K));
}

// Local diagonal of A_L at every point (closed form), to be assembled by QQ^T.
__global__ void local_diag_kernel(int N, int64_t L, const double* __restrict__ G,
                                  const double* __restrict__ D, double* __restrict__ d) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= L) return;
  const int N3 = N * N * N;
  const int64_t e = idx / N3;
  const int pt = (int)(idx - e * N3);
  const int i = pt % N, j = (pt / N) % N, k = pt / (N * N);
  const int64_t base = e * N3;
  const double* Grr = G;
  const double* Grs = G + L;
  const double* Grt = G + 2 * L;
  const double* Gss = G + 3 * L;
  const double* Gst = G + 4 * L;
  const double* Gtt = G + 5 * L;
  double v = 0.0;
  for (int l = 0; l < N; ++l) {
    const double a = D[l * N + i], b = D[l * N + j], c = D[l * N + k];
    v += a * a * Grr[base + l + N * (j + N * k)];
    v += b * b * Gss[base + i + N * (l + N * k)];
    v += c * c * Gtt[base + i + N * (j + N * l)];
  }
  const double Di = D[i * N + i], Dj = D[j * N + j], Dk = D[k * N + k];
  v += 2.0 * (Di * Dj * Grs[idx] + Di * Dk * Grt[idx] + Dj * Dk * Gst[idx]);
  d[idx] = v;
}

__global__ void invert_diag_kernel(int64_t L, const double* __restrict__ d,
                                   const uint8_t* __restrict__ pflag, double* __restrict__ dinv,
                                   float* __restrict__ dinv32) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= L) return;
  const double v = (pflag[idx] & PF_FREE) ? 1.0 / d[idx] : 0.0;
  dinv[idx] = v;
  if (dinv32) dinv32[idx] = (float)v;
}

__global__ void mass_times_kernel(int64_t L, const double* __restrict__ B,
                                  const double* __restrict__ f, double* __restrict__ b) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < L) b[idx] = B[idx] * f[idx];
}

__global__ void modes_rhs_kernel(int64_t L, const double* __restrict__ X, const double* __restrict__ B,
                                 int k1, int k2, int k3, double a, double* __restrict__ b) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= L) return;
  const double f = M_PI * M_PI * (double)(k1 * k1 + k2 * k2 + k3 * k3) * a *
                   sinpi(k1 * X[idx]) * sinpi(k2 * X[L + idx]) * sinpi(k3 * X[2 * L + idx]);
  b[idx] = B[idx] * f;
}

__global__ void diag_from_inv_kernel(int64_t L, const double* __restrict__ dinv,
                                     double* __restrict__ d) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < L) d[idx] = dinv[idx] != 0.0 ? 1.0 / dinv[idx] : 1.0;
}

template <class T>
__global__ void copy_cast_kernel(int64_t n, const double* __restrict__ a, T* __restrict__ b) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < n) b[idx] = (T)a[idx];
}

static int bc_mask_bits(const int bc[6]) {
  int m = 0;
  for (int f = 0; f < 6; ++f)
    if (bc[f] == SE_BC_DIRICHLET) m |= 1 << f;
  return m;
}

int build_level(se_mesh_s* m, int p, Level* lvp, Allocs& allocs, cudaStream_t s) {
  Level& lv = *lvp;
  lv.p = p;
  lv.N = p + 1;
  for (int d = 0; d < 3; ++d) lv.nel[d] = m->desc.nel[d];
  for (int f = 0; f < 6; ++f) lv.bc[f] = m->desc.bc[f];
  lv.E = (int64_t)lv.nel[0] * lv.nel[1] * lv.nel[2];
  const int N = lv.N, N3 = N * N * N;
  lv.L = lv.E * N3;
  lv.NX = lv.nel[0] * p + 1;
  lv.NY = lv.nel[1] * p + 1;
  SE_TRY(dmalloc(allocs, &lv.pstatus, 1));
  SE_TRY(dzero(lv.pstatus, sizeof(int), s));
  lv.NZ = lv.nel[2] * p + 1;
  lv.n_global = (int64_t)lv.NX * lv.NY * lv.NZ;
  SE_CHECK(lv.L < (int64_t)1 << 31, SE_EINVAL, "mesh too large: %lld local points (limit 2^31)",
           (long long)lv.L);
  lv.nbr = m->nbr;
  gll_basis(p, &lv.basis);
  double* dxi = nullptr;
  double* dw = nullptr;
  SE_TRY(dmalloc(allocs, &lv.D64, N * N));
  SE_TRY(dmalloc(allocs, &lv.D32, N * N));
  SE_TRY(dmalloc(allocs, &dxi, N));
  SE_TRY(dmalloc(allocs, &dw, N));
  float D32h[(SE_MAX_ORDER + 1) * (SE_MAX_ORDER + 1)];
  for (int t = 0; t < N * N; ++t) D32h[t] = (float)lv.basis.D[t];
  SE_TRY(h2d(lv.D64, lv.basis.D, N * N * sizeof(double), s));
  SE_TRY(h2d(lv.D32, D32h, N * N * sizeof(float), s));
  SE_TRY(h2d(dxi, lv.basis.xi, N * sizeof(double), s));
  SE_TRY(h2d(dw, lv.basis.w, N * sizeof(double), s));
  if (ax_eo_supported(p)) {
    const int H = N / 2;
    double tab[4 * (SE_MAX_ORDER + 1) * (SE_MAX_ORDER + 1) / 4 + 4];
    ax_eo_tables(lv.basis, tab);
    SE_TRY(dmalloc(allocs, &lv.eo64, 4 * H * H));
    SE_TRY(h2d(lv.eo64, tab, 4 * H * H * sizeof(double), s));
  }

  // geometry
  double* dverts = nullptr;
  const size_t nv = m->verts.size();
  SE_TRY(dmalloc(allocs, &dverts, nv));
  SE_TRY(h2d(dverts, m->verts.data(), nv * sizeof(double), s));
  SE_TRY(dmalloc(allocs, &lv.X, 3 * (size_t)lv.L));
  SE_TRY(dmalloc(allocs, &lv.G64, 6 * (size_t)lv.L));
  SE_TRY(dmalloc(allocs, &lv.B, (size_t)lv.L));
  const size_t smem = (3 * N3 + N * N) * sizeof(double);
  geometry_kernel<<<(unsigned)lv.E, N * N, smem, s>>>(N, lv.nel[0], lv.nel[1], dverts, dxi, dw,
                                                       lv.D64, m->desc.deform_amp, lv.L, lv.X,
                                                       lv.G64, lv.B);
  SE_LAUNCH_CHECK();
  SE_TRY(dmalloc(allocs, &lv.pflag, (size_t)lv.L));
  pointflag_kernel<<<grid_for(lv.L, 256), 256, 0, s>>>(N, lv.nel[0], lv.nel[1], lv.nel[2], lv.L,
                                                      bc_mask_bits(lv.bc), lv.pflag, nullptr);
  SE_LAUNCH_CHECK();
  if (m->desc.flags & SE_MESH_GS_MAP) SE_TRY(build_level_gsmap(lv, allocs, s));
  return SE_OK;
}

int build_jacobi(Level& lv, Allocs& allocs, Scratch& sc, cudaStream_t s) {
  (void)sc;
  double* d = nullptr;
  SE_TRY(dmalloc(allocs, &d, (size_t)lv.L));
  local_diag_kernel<<<grid_for(lv.L, 256), 256, 0, s>>>(lv.N, lv.L, lv.G64, lv.D64, d);
  SE_LAUNCH_CHECK();
  SE_TRY(gs_apply<double>(lv, d, false, s));
  SE_TRY(dmalloc(allocs, &lv.dinv64, (size_t)lv.L));
  SE_TRY(dmalloc(allocs, &lv.dinv32, (size_t)lv.L));
  invert_diag_kernel<<<grid_for(lv.L, 256), 256, 0, s>>>(lv.L, d, lv.pflag, lv.dinv64, lv.dinv32);
  SE_LAUNCH_CHECK();
  // the raw diagonal is no longer needed (freed in stream order after the inversion)
  dfree(allocs, d, (size_t)lv.L * sizeof(double));
  SE_CUDA(cudaStreamSynchronize(s));
  return SE_OK;
}

int local_to_global(const Level& lv, int* l2g, cudaStream_t s) {
  // recomputes the point flags identically and fills the global lattice id of every local point
  pointflag_kernel<<<grid_for(lv.L, 256), 256, 0, s>>>(lv.N, lv.nel[0], lv.nel[1], lv.nel[2], lv.L,
                                                      bc_mask_bits(lv.bc), lv.pflag, l2g);
  SE_LAUNCH_CHECK();
  return SE_OK;
}

int rhs_modes(se_mesh_s* m, const int k[3], double a, double* b, cudaStream_t s) {
  const Level& lv = m->fine;
  modes_rhs_kernel<<<grid_for(lv.L, 256), 256, 0, s>>>(lv.L, lv.X, lv.B, k[0], k[1], k[2], a, b);
  SE_LAUNCH_CHECK();
  return gs_apply<double>(lv, b, true, s);
}

int make_fp32_geometry(Level& lv, Allocs& allocs, cudaStream_t s) {
  if (lv.G32) return SE_OK;
  SE_TRY(dmalloc(allocs, &lv.G32, 6 * (size_t)lv.L));
  copy_cast_kernel<float><<<grid_for(6 * lv.L, 256), 256, 0, s>>>(6 * lv.L, lv.G64, lv.G32);
  SE_LAUNCH_CHECK();
  return SE_OK;
}

// Mean length of the 4 mapped corner-to-corner edges of each element along each direction
// (box-like approximation of Sec. 2.2.2, Fig. 1a).
static void box_lengths(se_mesh_s* m) {
  const int nx = m->desc.nel[0], ny = m->desc.nel[1], nz = m->desc.nel[2];
  const double amp = m->desc.deform_amp;
  const int64_t E = (int64_t)nx * ny * nz;
  m->box_len.assign(3 * E, 0.0);
  // every lattice vertex mapped once (a vertex is a corner of up to 8 elements)
  const int64_t nv = (int64_t)(nx + 1) * (ny + 1) * (nz + 1);
  std::vector<double> mapped(3 * nv);
  for (int64_t v = 0; v < nv; ++v) {
    const double* V = &m->verts[3 * v];
    const double sm = std::sin(2.0 * M_PI * V[0]) * std::sin(2.0 * M_PI * V[1]) *
                      std::sin(2.0 * M_PI * V[2]);
    for (int q = 0; q < 3; ++q) mapped[3 * v + q] = V[q] + amp * sm;
  }
  auto corner = [&](int a, int b, int c, double* x) {
    const int64_t v = a + (int64_t)(nx + 1) * (b + (int64_t)(ny + 1) * c);
    for (int q = 0; q < 3; ++q) x[q] = mapped[3 * v + q];
  };
  for (int64_t e = 0; e < E; ++e) {
    const int ex = (int)(e % nx), ey = (int)((e / nx) % ny), ez = (int)(e / ((int64_t)nx * ny));
    double C[2][2][2][3];
    for (int dz = 0; dz < 2; ++dz)
      for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx) corner(ex + dx, ey + dy, ez + dz, C[dz][dy][dx]);
    auto dist = [](const double* a, const double* b) {
      return std::sqrt((a[0] - b[0]) * (a[0] - b[0]) + (a[1] - b[1]) * (a[1] - b[1]) +
                       (a[2] - b[2]) * (a[2] - b[2]));
    };
    double lx = 0, ly = 0, lz = 0;
    for (int u = 0; u < 2; ++u)
      for (int v = 0; v < 2; ++v) {
        lx += dist(C[u][v][1], C[u][v][0]);
        ly += dist(C[u][1][v], C[u][0][v]);
        lz += dist(C[1][u][v], C[0][u][v]);
      }
    m->box_len[3 * e + 0] = lx / 4.0;
    m->box_len[3 * e + 1] = ly / 4.0;
    m->box_len[3 * e + 2] = lz / 4.0;
  }
}

}  // namespace se

using namespace se;

extern "C" {

int se_mesh_create(const se_mesh_desc* desc, se_mesh_t* out) {
  SE_CHECK(desc && out, SE_EINVAL, "se_mesh_create: null argument");
  SE_CHECK(desc->p >= 1 && desc->p <= SE_MAX_ORDER, SE_EINVAL, "se_mesh_create: p=%d not in 1..%d",
           desc->p, SE_MAX_ORDER);
  for (int d = 0; d < 3; ++d)
    SE_CHECK(desc->nel[d] >= 1, SE_EINVAL, "se_mesh_create: nel[%d]=%d < 1", d, desc->nel[d]);
  for (int f = 0; f < 6; ++f)
    SE_CHECK(desc->bc[f] == SE_BC_DIRICHLET || desc->bc[f] == SE_BC_NEUMANN, SE_EINVAL,
             "se_mesh_create: bad bc[%d]", f);
  auto* m = new se_mesh_s();
  m->desc = *desc;
  m->desc.vertex_xyz = nullptr;
  const int nx = desc->nel[0], ny = desc->nel[1], nz = desc->nel[2];
  const int64_t nv = (int64_t)(nx + 1) * (ny + 1) * (nz + 1);
  m->verts.resize(3 * nv);
  if (desc->vertex_xyz) {
    std::memcpy(m->verts.data(), desc->vertex_xyz, 3 * nv * sizeof(double));
  } else {
    const double h[3] = {1.0 / nx, 1.0 / ny, 1.0 / nz};
    for (int c = 0; c <= nz; ++c)
      for (int b = 0; b <= ny; ++b)
        for (int a = 0; a <= nx; ++a) {
          const int64_t v = a + (int64_t)(nx + 1) * (b + (int64_t)(ny + 1) * c);
          const double x0[3] = {(double)a / nx, (double)b / ny, (double)c / nz};
          const bool interior = a > 0 && a < nx && b > 0 && b < ny && c > 0 && c < nz;
          for (int d = 0; d < 3; ++d) {
            double x = x0[d];
            if (interior && desc->perturb_frac != 0.0)
              x += desc->perturb_frac * h[d] * (2.0 * uniform01(desc->seed, 3 * (uint64_t)v + d) - 1.0);
            m->verts[3 * v + d] = x;
          }
        }
  }
  int st = SE_OK;
  auto fail = [&](int code) {
    m->allocs.release();
    if (m->stream) cudaStreamDestroy(m->stream);
    pinned_release(m->scratch.hscal);
    delete m;
    return code;
  };
  const unsigned sflags = (desc->flags & SE_MESH_NONBLOCKING_STREAM) ? cudaStreamNonBlocking : cudaStreamDefault;
  if (cudaStreamCreateWithFlags(&m->stream, sflags) != cudaSuccess) {
    set_error("se_mesh_create: cudaStreamCreate failed");
    return fail(SE_ECUDA);
  }
  m->allocs.stream = m->stream;
  if ((st = scratch_alloc(m->allocs, &m->scratch)) != SE_OK) return fail(st);
  // element neighbours, offsets (dx, dy, dz) in {-1,0,1}^3 at slot (dx+1) + 3(dy+1) + 9(dz+1)
  const int64_t E = (int64_t)nx * ny * nz;
  {
    std::vector<int> nb(27 * E);
    for (int64_t e = 0; e < E; ++e) {
      const int ex = (int)(e % nx), ey = (int)((e / nx) % ny), ez = (int)(e / ((int64_t)nx * ny));
      for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
          for (int dx = -1; dx <= 1; ++dx) {
            const int a = ex + dx, b = ey + dy, c = ez + dz;
            const bool ok = a >= 0 && a < nx && b >= 0 && b < ny && c >= 0 && c < nz;
            nb[27 * e + (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1)] =
                ok ? (int)(a + (int64_t)nx * (b + (int64_t)ny * c)) : -1;
          }
    }
    if ((st = dmalloc(m->allocs, &m->nbr, nb.size())) != SE_OK) return fail(st);
    if ((st = h2d(m->nbr, nb.data(), nb.size() * sizeof(int), m->stream)) != SE_OK) return fail(st);
  }
  box_lengths(m);
  if ((st = build_level(m, desc->p, &m->fine, m->allocs, m->stream)) != SE_OK) return fail(st);
  if ((st = build_jacobi(m->fine, m->allocs, m->scratch, m->stream)) != SE_OK) return fail(st);
  if ((st = dmalloc(m->allocs, &m->tmp64, (size_t)m->fine.L)) != SE_OK) return fail(st);
  if ((st = dmalloc(m->allocs, &m->tmpa32, (size_t)m->fine.L)) != SE_OK) return fail(st);
  if ((st = dmalloc(m->allocs, &m->tmpb32, (size_t)m->fine.L)) != SE_OK) return fail(st);
  if (cudaStreamSynchronize(m->stream) != cudaSuccess) {
    set_error("se_mesh_create: %s", cudaGetErrorString(cudaGetLastError()));
    return fail(SE_ECUDA);
  }
  *out = m;
  return SE_OK;
}

int se_mesh_destroy(se_mesh_t m) {
  if (!m) return SE_OK;
  cudaStreamSynchronize(m->stream);
  if (m->gexec) cudaGraphExecDestroy(m->gexec);
  if (m->ev0) cudaEventDestroy(m->ev0);
  if (m->ev1) cudaEventDestroy(m->ev1);
  m->allocs.release();
  pinned_release(m->scratch.hscal);
  cudaStreamDestroy(m->stream);
  delete m;
  return SE_OK;
}

int se_mesh_get_info(se_mesh_t m, se_mesh_info* info) {
  SE_CHECK(m && info, SE_EINVAL, "se_mesh_get_info: null argument");
  const Level& lv = m->fine;
  info->E = lv.E;
  info->N = lv.N;
  info->L = lv.L;
  info->n_global = lv.n_global;
  info->n_dof = lv.E * (int64_t)lv.p * lv.p * lv.p;
  info->p = lv.p;
  for (int d = 0; d < 3; ++d) info->nel[d] = lv.nel[d];
  return SE_OK;
}

int se_mesh_nodes(se_mesh_t m, double* xyz_dev, void* stream) {
  SE_CHECK(m && xyz_dev, SE_EINVAL, "se_mesh_nodes: null argument");
  SE_CUDA(cudaMemcpyAsync(xyz_dev, m->fine.X, 3 * (size_t)m->fine.L * sizeof(double),
                          cudaMemcpyDeviceToDevice, as_stream(stream, m->stream)));
  return SE_OK;
}

int se_mesh_vertices(se_mesh_t m, double* xyz_host) {
  SE_CHECK(m && xyz_host, SE_EINVAL, "se_mesh_vertices: null argument");
  std::memcpy(xyz_host, m->verts.data(), m->verts.size() * sizeof(double));
  return SE_OK;
}

int se_mesh_rhs(se_mesh_t m, const double* f_dev, double* b_dev, void* stream) {
  SE_CHECK(m && f_dev && b_dev, SE_EINVAL, "se_mesh_rhs: null argument");
  cudaStream_t s = as_stream(stream, m->stream);
  const Level& lv = m->fine;
  mass_times_kernel<<<grid_for(lv.L, 256), 256, 0, s>>>(lv.L, lv.B, f_dev, b_dev);
  SE_LAUNCH_CHECK();
  return gs_apply<double>(lv, b_dev, true, s);
}

int se_jacobi_diag(se_mesh_t m, double* d_dev, void* stream) {
  SE_CHECK(m && d_dev, SE_EINVAL, "se_jacobi_diag: null argument");
  cudaStream_t s = as_stream(stream, m->stream);
  diag_from_inv_kernel<<<grid_for(m->fine.L, 256), 256, 0, s>>>(m->fine.L, m->fine.dinv64, d_dev);
  SE_LAUNCH_CHECK();
  return SE_OK;
}

}  // extern "C"
