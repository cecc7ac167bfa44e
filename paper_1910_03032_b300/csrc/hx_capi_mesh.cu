// C ABI of libhx.so (include/hx.h): errors, mesh and restriction set-up (Sec. 3, Sec. 3.1).
#include "hx_capi_internal.h"

using namespace hxc;

namespace hxc {

namespace {
thread_local std::string g_err;
}  // namespace

std::string& last_error() { return g_err; }

hx_status fail(hx_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

hx_status cuda_fail(cudaError_t e, const char* what) {
  cudaGetLastError();  // clear a non-sticky error
  if (e == cudaErrorMemoryAllocation) return fail(HX_ERR_OOM, "%s: out of device memory", what);
  return fail(HX_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

}  // namespace hxc

void hx_internal_set_error(const char* msg) { hxc::last_error() = msg; }

namespace hxc {

hx_apply_launcher apply_launcher(int p) {
  static const hx_apply_launcher t[] = {nullptr, hx_launch_apply_p1, hx_launch_apply_p2, hx_launch_apply_p3,
                                        hx_launch_apply_p4, hx_launch_apply_p5, hx_launch_apply_p6,
                                        hx_launch_apply_p7, hx_launch_apply_p8};
  return t[p];
}
hx_diag_launcher diag_launcher(int p) {
  static const hx_diag_launcher t[] = {nullptr, hx_launch_diag_p1, hx_launch_diag_p2, hx_launch_diag_p3,
                                       hx_launch_diag_p4, hx_launch_diag_p5, hx_launch_diag_p6,
                                       hx_launch_diag_p7, hx_launch_diag_p8};
  return t[p];
}
hx_load_launcher load_launcher(int p) {
  static const hx_load_launcher t[] = {nullptr, hx_launch_load_p1, hx_launch_load_p2, hx_launch_load_p3,
                                       hx_launch_load_p4, hx_launch_load_p5, hx_launch_load_p6,
                                       hx_launch_load_p7, hx_launch_load_p8};
  return t[p];
}

hx_status check_order(int p, int q) {
  if (p < 1 || p > HX_PMAX) return fail(HX_ERR_UNSUPPORTED, "p = %d outside 1..%d", p, HX_PMAX);
  if (q != p + 1 && q != p + 2) return fail(HX_ERR_UNSUPPORTED, "q = %d not in {p+1, p+2} for p = %d", q, p);
  return HX_OK;
}

// Build the device mesh from host arrays.  restriction is [E][n^3] int64.
hx_status build_mesh(int p, int q, long long n_vert, const double* vert, long long E, const int64_t* ev,
                     long long n_dof, const int64_t* R, const uint8_t* dir, hx_mesh** out) {
  const int n = p + 1, N3 = n * n * n;
  if ((long double)E * N3 >= 2147483647.0L)
    return fail(HX_ERR_UNSUPPORTED, "n_elem * (p+1)^3 = %lld exceeds int32 indexing", (long long)E * N3);
  if (n_dof >= 2147483647LL) return fail(HX_ERR_UNSUPPORTED, "n_dof too large");
  // host-side restriction encoding and transpose (counting sort: deterministic order)
  std::vector<int> Renc((size_t)E * N3);
  std::vector<int> off((size_t)n_dof + 1, 0);
  for (long long k = 0; k < E * N3; ++k) {
    const long long g = R[k];
    if (g < 0 || g >= n_dof) return fail(HX_ERR_ARG, "restriction entry %lld = %lld outside [0, %lld)", k, g, n_dof);
    off[g + 1] += 1;
  }
  for (long long g = 0; g < n_dof; ++g) {
    if (off[g + 1] == 0) return fail(HX_ERR_ARG, "global DoF %lld belongs to no element", g);
    off[g + 1] += off[g];
  }
  std::vector<int> idx((size_t)E * N3), fill(off.begin(), off.end() - 1);
  for (long long k = 0; k < E * N3; ++k) {
    const long long g = R[k];
    idx[fill[g]++] = (int)k;
    Renc[k] = (dir && dir[g]) ? (int)(-g - 1) : (int)g;
  }
  std::vector<double> X8((size_t)E * 24);
  for (long long e = 0; e < E; ++e)
    for (int c = 0; c < 8; ++c) {
      const long long v = ev[e * 8 + c];
      if (v < 0 || v >= n_vert) return fail(HX_ERR_ARG, "elem_vert[%lld][%d] = %lld out of range", e, c, v);
      for (int d = 0; d < 3; ++d) X8[e * 24 + c * 3 + d] = vert[v * 3 + d];
    }
  std::vector<unsigned char> dmask((size_t)n_dof, 0);
  if (dir)
    for (long long g = 0; g < n_dof; ++g) dmask[g] = dir[g] ? 1 : 0;

  hx_mesh* m = new (std::nothrow) hx_mesh();
  if (!m) return fail(HX_ERR_OOM, "host allocation failed");
  m->p = p;
  m->q = q;
  m->n = n;
  m->N3 = N3;
  m->E = E;
  m->n_dof = n_dof;
  for (long long g = 0; g < n_dof; ++g) m->n_dirichlet += dmask[g];
  cudaGetDevice(&m->device);
  if (hx_build_tables(p, q, &m->T) == 0) hx_tables_to_float(m->T, &m->T32);
  else {
    delete m;
    return fail(HX_ERR_UNSUPPORTED, "cannot build tables for p=%d q=%d", p, q);
  }
  hx_status s;
  // 4 ints of slack: the FP32 kernel's bulk copies of restriction ranges round their end up to 16 bytes
  if ((s = dalloc(&m->R, Renc.size() + 4, "mesh restriction")) || (s = dalloc(&m->off, off.size(), "mesh offsets")) ||
      (s = dalloc(&m->idx, idx.size(), "mesh transpose")) || (s = dalloc(&m->dir, dmask.size(), "mesh mask")) ||
      (s = dalloc(&m->X8, X8.size(), "mesh vertices"))) {
    hx_mesh_destroy(m);
    return s;
  }
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = cudaMemcpy(m->R, Renc.data(), Renc.size() * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(m->off, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(m->idx, idx.data(), idx.size() * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(m->dir, dmask.data(), dmask.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(m->X8, X8.data(), X8.size() * sizeof(double), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    hx_mesh_destroy(m);
    return cuda_fail(e, "mesh upload");
  }
  *out = m;
  return HX_OK;
}

}  // namespace hxc

extern "C" {

int hx_version(void) { return 100; }

const char* hx_last_error(void) { return hxc::last_error().c_str(); }

hx_status hx_mesh_create(int p, int q, int64_t n_vert, const double* vert_xyz, int64_t n_elem,
                         const int64_t* elem_vert, int64_t n_dof, const int64_t* restriction, const uint8_t* dirichlet,
                         hx_mesh** out) {
  if (!out) return fail(HX_ERR_ARG, "out is NULL");
  *out = nullptr;
  hx_status s = check_order(p, q);
  if (s) return s;
  if (n_vert < 8 || n_elem < 1 || n_dof < 1 || !vert_xyz || !elem_vert || !restriction)
    return fail(HX_ERR_ARG, "bad sizes or NULL arrays");
  return build_mesh(p, q, n_vert, vert_xyz, n_elem, elem_vert, n_dof, restriction, dirichlet, out);
}

hx_status hx_mesh_create_box(int nx, int ny, int nz, int p, int q, const double* vert_xyz, int dirichlet_faces,
                             hx_mesh** out) {
  if (!out) return fail(HX_ERR_ARG, "out is NULL");
  *out = nullptr;
  hx_status s = check_order(p, q);
  if (s) return s;
  if (nx < 1 || ny < 1 || nz < 1 || !vert_xyz) return fail(HX_ERR_ARG, "bad grid size or NULL vertices");
  const int n = p + 1, N3 = n * n * n;
  const long long E = (long long)nx * ny * nz;
  const long long gx = (long long)p * nx + 1, gy = (long long)p * ny + 1, gz = (long long)p * nz + 1;
  const long long n_dof = gx * gy * gz;
  if ((long double)E * N3 >= 2147483647.0L) return fail(HX_ERR_UNSUPPORTED, "mesh too large for int32 indexing");
  const long long n_vert = (long long)(nx + 1) * (ny + 1) * (nz + 1);
  std::vector<int64_t> ev((size_t)E * 8), R((size_t)E * N3);
  std::vector<uint8_t> dir((size_t)n_dof);
  const long long sx = nx + 1, sy = (long long)(nx + 1) * (ny + 1);
  long long e = 0;
  for (int ez = 0; ez < nz; ++ez)
    for (int ey = 0; ey < ny; ++ey)
      for (int ex = 0; ex < nx; ++ex, ++e) {
        for (int c = 0; c < 8; ++c)
          ev[e * 8 + c] = (ex + (c & 1)) + (ey + ((c >> 1) & 1)) * sx + (ez + ((c >> 2) & 1)) * sy;
        int l = 0;
        for (int k = 0; k < n; ++k)
          for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i, ++l)
              R[e * N3 + l] = ((long long)p * ex + i) + gx * (((long long)p * ey + j) + gy * ((long long)p * ez + k));
      }
  long long g = 0;
  for (long long K = 0; K < gz; ++K)
    for (long long J = 0; J < gy; ++J)
      for (long long I = 0; I < gx; ++I, ++g)
        dir[g] = (((dirichlet_faces & 1) && I == 0) || ((dirichlet_faces & 2) && I == gx - 1) ||
                  ((dirichlet_faces & 4) && J == 0) || ((dirichlet_faces & 8) && J == gy - 1) ||
                  ((dirichlet_faces & 16) && K == 0) || ((dirichlet_faces & 32) && K == gz - 1))
                     ? 1
                     : 0;
  s = build_mesh(p, q, n_vert, vert_xyz, E, ev.data(), n_dof, R.data(), dir.data(), out);
  if (s == HX_OK) {
    (*out)->grid[0] = gx;
    (*out)->grid[1] = gy;
    (*out)->grid[2] = gz;
    (*out)->ga = hx_grid_asm(p, nx, ny, nz, (int)gx, (int)gy);
    (*out)->lay = hx_elayout_rows(nx);
  }
  return s;
}

hx_status hx_mesh_create_structured(int nx, int ny, int nz, int p, int q, const double* vert_xyz, hx_mesh** out) {
  return hx_mesh_create_box(nx, ny, nz, p, q, vert_xyz, 63, out);
}

void hx_mesh_destroy(hx_mesh* m) {
  if (!m) return;
  dfree(m->R);
  dfree(m->off);
  dfree(m->idx);
  dfree(m->dir);
  dfree(m->X8);
  delete m;
}

hx_status hx_mesh_info(const hx_mesh* m, int64_t* n_elem, int64_t* n_dof, int* p, int* q) {
  if (!m) return fail(HX_ERR_ARG, "mesh is NULL");
  if (n_elem) *n_elem = m->E;
  if (n_dof) *n_dof = m->n_dof;
  if (p) *p = m->p;
  if (q) *q = m->q;
  return HX_OK;
}

hx_status hx_mesh_qpoint_coords(const hx_mesh* m, double* xyz, void* stream) {
  if (!m || !xyz) return fail(HX_ERR_ARG, "NULL argument");
  HX_TRY(hx_launch_qpoint_coords(m->T, m->E, m->X8, xyz, (cudaStream_t)stream), "qpoint coords");
  return HX_OK;
}

hx_status hx_mesh_node_coords(const hx_mesh* m, double* xyz, void* stream) {
  if (!m || !xyz) return fail(HX_ERR_ARG, "NULL argument");
  HX_TRY(hx_launch_node_coords(m->T, m->n_dof, m->off, m->idx, m->X8, xyz, (cudaStream_t)stream), "node coords");
  return HX_OK;
}

}  // extern "C"
