// libdg host runtime: C-ABI entry points (include/dg.h), mesh validation and
// face matching, element geometry, reference tables, state conversion,
// sources/receivers, and the step loop that enqueues the CUDA kernels.
#include "../../include/dg.h"

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <unordered_map>
#include <vector>

#include "dg_internal.h"
#include "dg_reference.h"
#include "dg_revolve.h"

using namespace dg;

namespace {

thread_local std::string g_last_error;

struct FaceKey {
  int64_t a, b, c;
  bool operator==(const FaceKey& o) const { return a == o.a && b == o.b && c == o.c; }
};
struct FaceKeyHash {
  size_t operator()(const FaceKey& k) const {
    uint64_t h = 1469598103934665603ull;
    for (int64_t v : {k.a, k.b, k.c}) {
      h ^= static_cast<uint64_t>(v) + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2);
      h *= 1099511628211ull;
    }
    return static_cast<size_t>(h);
  }
};

// dg_step_host streams the state through the device in element chunks, whose
// boundaries (multiples of 16 elements) this returns: about 1/16 of the elements in
// the first chunk and in the last, whose upload and download nothing hides, and the
// rest in seven equal chunks; at least 4096 elements per chunk, so small meshes take
// fewer (more than about nine chunks measured slower).
std::vector<int64_t> host_chunk_bounds(int64_t E) {
  auto r16 = [](int64_t x) { return (x + 15) / 16 * 16; };
  std::vector<int64_t> b{0};
  const int64_t edge = r16(std::max<int64_t>(4096, E / 16));
  if (E <= 2 * edge + 4096) {                 // uniform chunks of at least 4096
    const int64_t chunk = r16(std::max<int64_t>(4096, (E + 7) / 8));
    for (int64_t e = chunk; e < E; e += chunk) b.push_back(e);
  } else {
    const int64_t last = (E - edge) / 16 * 16;  // start of the last chunk
    b.push_back(edge);
    const int64_t mid = last - edge;
    const int64_t parts = std::max<int64_t>(1, std::min<int64_t>(7, mid / 4096));
    const int64_t chunk = r16((mid + parts - 1) / parts);
    for (int64_t e = edge + chunk; e < last; e += chunk) b.push_back(e);
    b.push_back(last);
  }
  b.push_back(E);
  return b;
}

// the chunk of element e
int host_chunk_of(const std::vector<int64_t>& b, int64_t e) {
  return static_cast<int>(std::upper_bound(b.begin(), b.end(), e) - b.begin()) - 1;
}

// The faces of one such chunk: the interior faces first seen from its elements
// (the flux list holds them in ascending order of that element), the last chunk
// whose predictor they read (the other side's chunk), and its boundary faces.
struct HostChunkFaces {
  int64_t fi0 = 0, fi1 = 0;
  int64_t fb0 = 0, fb1 = 0;
  int need = 0;
};

}  // namespace

struct dg_ctx {
  int N = 0, L = 0, M = 1;
  int law = 0;                       // 0 = CDM, 1 = IVM, 2 = nonlinear shear
  int picard_iters = 0;              // Picard iterations after the CK predictor (0: CK alone)
  int wait_limit = -1;               // polls of the tensor-core waits (-1: the kernels' default)
  int64_t E = 0;                     // mesh elements
  int64_t EV = 0;                    // element copies on the device: E x members, member fastest
  double cfl = 0.5;
  cudaStream_t stream = nullptr;
  dg_allocator alloc{};
  bool has_alloc = false;
  std::string err;

  // host copies (sorted vertex order)
  std::vector<double> xyz_user;      // [E][4][3] as given
  std::vector<double> xyz;           // [E][4][3] vertices by increasing vertex id
  std::vector<double> jinv;          // [E][9] Theta^{-1} of the sorted order
  std::vector<double> detj;          // [E] |det J|
  std::vector<double> rin;           // [E] inradius
  std::vector<double> mat;           // [E][6] (member 0's xi0 and C_d when members > 1)
  bool has_material = false, has_state = false;
  double dt_cfl = 0.0, t = 0.0;

  // device memory
  float* q[2] = {nullptr, nullptr};
  int cur = 0;
  float* d = nullptr;
  float* cp = nullptr;
  float* ff = nullptr;               // face fluxes
  int4* faces = nullptr;
  int* elem_face = nullptr;
  int64_t F = 0;            // faces in the flux list: interior first, then boundary
  int64_t F_interior = 0;
  int grid_pred = 0, grid_face = 0, grid_corr = 0;
  cudaStream_t copy_stream = nullptr;     // host transfers of dg_step_host (created on first use)
  std::vector<cudaEvent_t> xfer_events;   // [2 x chunks + 1] for dg_step_host
  std::vector<HostChunkFaces> host_faces;  // per chunk of dg_step_host (one member only)
  GeomF* geom = nullptr;
  MatF* matf = nullptr;
  int* nbr = nullptr;
  float* tables = nullptr;
  unsigned* status = nullptr;
  void* staging = nullptr;
  size_t staging_bytes = 0;
  unsigned* status_host = nullptr;   // pinned

  // sources
  std::vector<dg_point_source> sources;
  std::vector<SourceDev> source_host;   // sources x members (member fastest)
  SourceDev* source_dev = nullptr;
  float* amp_dev = nullptr;
  int64_t amp_cap = 0;
  float* amp_host = nullptr;         // pinned

  // receivers
  std::vector<ReceiverDev> rec_host;    // members x receivers (receiver fastest)
  ReceiverDev* rec_dev = nullptr;
  float* traces = nullptr;
  int64_t trace_cap = 0, n_rec = 0;

  // stats / profiling
  dg_stats stats{};
  bool profiling = false;
  std::vector<cudaEvent_t> events;
  std::vector<int> event_kind;
  dg_kernel_time prof[5]{};

  std::vector<std::pair<void*, size_t>> owned;

  // point location: uniform buckets over the element bounding boxes (built on first use)
  double bb_lo[3] = {0, 0, 0}, bb_cell[3] = {1, 1, 1};
  int bb_n[3] = {0, 0, 0};
  std::vector<int64_t> bucket_start, bucket_elems;
};

namespace {

dg_status fail(dg_ctx* ctx, dg_status s, const std::string& msg) {
  if (ctx) ctx->err = msg;
  g_last_error = msg;
  return s;
}

dg_status cuda_fail(dg_ctx* ctx, cudaError_t e, const char* what) {
  return fail(ctx, DG_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define DG_CUDA(ctx, call)                                   \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
  } while (0)

void* dev_alloc(dg_ctx* ctx, size_t bytes) {
  if (bytes == 0) bytes = 16;
  void* p = nullptr;
  if (ctx->has_alloc) {
    p = ctx->alloc.alloc(bytes, ctx->stream, ctx->alloc.user);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) ctx->owned.emplace_back(p, bytes);
  return p;
}

void dev_free(dg_ctx* ctx, void* p) {
  if (!p) return;
  for (size_t i = 0; i < ctx->owned.size(); ++i) {
    if (ctx->owned[i].first == p) {
      if (ctx->has_alloc) ctx->alloc.free(p, ctx->owned[i].second, ctx->stream, ctx->alloc.user);
      else cudaFree(p);
      ctx->owned.erase(ctx->owned.begin() + i);
      return;
    }
  }
}

bool supported_order(int N) { return N >= 1 && N <= kMaxOrder; }

void inv3(const double* J, double* out, double* det) {
  // J row-major 3x3; out = J^{-1}
  const double a = J[0], b = J[1], c = J[2], d = J[3], e = J[4], f = J[5], g = J[6], h = J[7], i = J[8];
  const double A = e * i - f * h, B = -(d * i - f * g), C = d * h - e * g;
  const double D = det[0] = a * A + b * B + c * C;
  out[0] = A / D; out[1] = -(b * i - c * h) / D; out[2] = (b * f - c * e) / D;
  out[3] = B / D; out[4] = (a * i - c * g) / D;  out[5] = -(a * f - c * d) / D;
  out[6] = C / D; out[7] = -(a * h - b * g) / D; out[8] = (a * e - b * d) / D;
}

// Round an FP32 value to the nearest TF32 value (10 mantissa bits), ties away
// from zero, as the tensor cores' conversion does.
float tf32_round(float x) {
  uint32_t u;
  std::memcpy(&u, &x, 4);
  if ((u & 0x7F800000u) != 0x7F800000u) {
    u += 0x1000u;
    u &= 0xFFFFE000u;
  }
  float r;
  std::memcpy(&r, &u, 4);
  return r;
}

// Reference tables of degree N (FP64), in the layout of table_layout(N).
std::vector<double> build_tables(int N) {
  const int L = n_modes(N), NQ = n_vol_nodes(N), NF = n_face_nodes(N), NT = N + 1;
  const int LP = lp_of(N), NQP = nqp_of(N), NFP = nfp_of(N);
  const TableLayout T = table_layout(N);
  std::vector<double> t(T.total, 0.0);
  ref::Rule3 vr = ref::volume_rule(N + 1);
  std::vector<double> val(L), grd(3 * L);
  std::vector<double> Kt(3 * L * L, 0.0);   // Kt[e][k][l] = int phi_k d phi_l / d xi_e
  for (int q = 0; q < NQ; ++q) {
    ref::dubiner(N, vr.xi[q], vr.eta[q], vr.zeta[q], val.data(), grd.data());
    for (int l = 0; l < L; ++l) {
      t[T.VvT + l * NQP + q] = val[l];
      t[T.Vw + q * LP + l] = vr.w[q] * val[l];
      for (int e = 0; e < 3; ++e) t[T.Gw + (e * NQ + q) * LP + l] = vr.w[q] * grd[3 * l + e];
    }
    // the rule is exact for the degree 2N-1 integrands of Kt
    for (int e = 0; e < 3; ++e)
      for (int k = 0; k < L; ++k)
        for (int l = 0; l < L; ++l) Kt[(e * L + k) * L + l] += vr.w[q] * val[k] * grd[3 * l + e];
  }
  for (int e = 0; e < 3; ++e)
    for (int k = 0; k < L; ++k)
      for (int l = 0; l < L; ++l) {
        t[T.KtA + (e * L + l) * LP + k] = Kt[(e * L + k) * L + l];
        t[T.KtB + (e * L + k) * LP + l] = Kt[(e * L + k) * L + l];
      }
  ref::Rule2 fr = ref::face_rule(N + 1);
  const double R[4][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
  for (int f = 0; f < 4; ++f) {
    int v[3], n = 0;
    for (int j = 0; j < 4; ++j) if (j != f) v[n++] = j;
    for (int i = 0; i < NF; ++i) {
      double p[3];
      for (int c = 0; c < 3; ++c)
        p[c] = R[v[0]][c] + fr.s[i] * (R[v[1]][c] - R[v[0]][c]) + fr.t[i] * (R[v[2]][c] - R[v[0]][c]);
      ref::dubiner(N, p[0], p[1], p[2], val.data(), nullptr);
      for (int l = 0; l < L; ++l) {
        t[T.VfT + (f * L + l) * NFP + i] = val[l];
        t[T.Vfw + (f * NF + i) * LP + l] = fr.w[i] * val[l];
      }
    }
  }
  if (tc_volume(N)) {
    const int KP = tc_kp(N);
    for (int q = 0; q < NQ; ++q)
      for (int l = 0; l < L; ++l) {
        const float x = static_cast<float>(t[T.VvT + l * NQP + q]);
        const float h = tf32_round(x);
        t[T.PhiH + tc_canon(q, l, KP)] = h;
        t[T.PhiL + tc_canon(q, l, KP)] = tf32_round(x - h);
      }
    const int KQ = tc_kq(N);
    for (int l = 0; l < L; ++l)
      for (int q = 0; q < NQ; ++q) {
        const float x = static_cast<float>(t[T.Vw + q * LP + l]);
        const float h = tf32_round(x);
        t[T.PrjH + l * KQ + q] = h;
        t[T.PrjL + l * KQ + q] = tf32_round(x - h);
      }
    for (int l = 0; l < L; ++l) {
      double sum = 0.0;
      for (int q = 0; q < NQ; ++q) sum += t[T.Vw + q * LP + l];
      t[T.PrjS + l] = sum;
    }
  }
  ref::Rule1 tr = ref::time_rule(NT);
  for (int z = 0; z < NT; ++z) {
    t[T.tz + z] = tr.x[z];
    t[T.gz + z] = tr.w[z];
  }
  // Tfit = V^{-1}, V[z][j] = tz_z^j / j!, by Gauss-Jordan elimination with partial pivoting
  {
    std::vector<double> A(NT * 2 * NT, 0.0);
    for (int z = 0; z < NT; ++z) {
      double p = 1.0, f = 1.0;
      for (int j = 0; j < NT; ++j) {
        A[z * 2 * NT + j] = p / f;
        p *= tr.x[z];
        f *= (j + 1);
      }
      A[z * 2 * NT + NT + z] = 1.0;
    }
    for (int c = 0; c < NT; ++c) {
      int piv = c;
      for (int r = c + 1; r < NT; ++r)
        if (std::fabs(A[r * 2 * NT + c]) > std::fabs(A[piv * 2 * NT + c])) piv = r;
      for (int k = 0; k < 2 * NT; ++k) std::swap(A[c * 2 * NT + k], A[piv * 2 * NT + k]);
      const double d = A[c * 2 * NT + c];
      for (int k = 0; k < 2 * NT; ++k) A[c * 2 * NT + k] /= d;
      for (int r = 0; r < NT; ++r) {
        if (r == c) continue;
        const double m = A[r * 2 * NT + c];
        for (int k = 0; k < 2 * NT; ++k) A[r * 2 * NT + k] -= m * A[c * 2 * NT + k];
      }
    }
    for (int j = 0; j < NT; ++j)
      for (int z = 0; z < NT; ++z) t[T.Tfit + j * NT + z] = A[j * 2 * NT + NT + z];
  }
  return t;
}

template <typename T>
dg_status upload(dg_ctx* ctx, T* dst, const void* src, size_t bytes) {
  DG_CUDA(ctx, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, ctx->stream));
  DG_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return DG_OK;
}

// first element (input order) whose closure contains x; fills xi in the sorted order
void build_buckets(dg_ctx* ctx) {
  const int64_t E = ctx->E;
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int64_t i = 0; i < 4 * E; ++i)
    for (int c = 0; c < 3; ++c) {
      lo[c] = std::min(lo[c], ctx->xyz_user[3 * i + c]);
      hi[c] = std::max(hi[c], ctx->xyz_user[3 * i + c]);
    }
  // about one bucket per element, shaped like the mesh's bounding box
  double ext[3], vol = 1.0;
  for (int c = 0; c < 3; ++c) {
    ext[c] = std::max(hi[c] - lo[c], 1e-300);
    vol *= ext[c];
  }
  const double cell = std::cbrt(vol / static_cast<double>(std::max<int64_t>(E, 1)));
  int64_t total = 1;
  for (int c = 0; c < 3; ++c) {
    ctx->bb_n[c] = static_cast<int>(std::min<double>(std::max(1.0, std::ceil(ext[c] / cell)), 2048.0));
    ctx->bb_lo[c] = lo[c];
    ctx->bb_cell[c] = ext[c] / ctx->bb_n[c];
    total *= ctx->bb_n[c];
  }
  auto range = [&](int64_t e, int lo_i[3], int hi_i[3]) {
    for (int c = 0; c < 3; ++c) {
      double a = INFINITY, b = -INFINITY;
      for (int v = 0; v < 4; ++v) {
        a = std::min(a, ctx->xyz_user[12 * e + 3 * v + c]);
        b = std::max(b, ctx->xyz_user[12 * e + 3 * v + c]);
      }
      const double pad = 1e-9 * (b - a) + 1e-300;
      lo_i[c] = std::max(0, static_cast<int>(std::floor((a - pad - ctx->bb_lo[c]) / ctx->bb_cell[c])));
      hi_i[c] = std::min(ctx->bb_n[c] - 1, static_cast<int>(std::floor((b + pad - ctx->bb_lo[c]) / ctx->bb_cell[c])));
    }
  };
  std::vector<int64_t> count(total + 1, 0);
  for (int pass = 0; pass < 2; ++pass) {
    if (pass == 1) {
      for (int64_t i = 0; i < total; ++i) count[i + 1] += count[i];
      ctx->bucket_start = count;
      ctx->bucket_elems.assign(count[total], 0);
    }
    std::vector<int64_t> fill;
    if (pass == 1) fill.assign(ctx->bucket_start.begin(), ctx->bucket_start.end() - 1);
    for (int64_t e = 0; e < E; ++e) {           // ascending element order within each bucket
      int a[3], b[3];
      range(e, a, b);
      for (int i = a[0]; i <= b[0]; ++i)
        for (int j = a[1]; j <= b[1]; ++j)
          for (int k = a[2]; k <= b[2]; ++k) {
            const int64_t id = (static_cast<int64_t>(k) * ctx->bb_n[1] + j) * ctx->bb_n[0] + i;
            if (pass == 0) ++count[id + 1];
            else ctx->bucket_elems[fill[id]++] = e;
          }
    }
  }
}

// The first element (input order) whose closure contains x, and x in that
// element's reference coordinates of the sorted vertex order.
bool locate(dg_ctx* ctx, const double* x, int64_t* elem, double xi_sorted[3]) {
  const double tol = 1e-10;
  if (ctx->bucket_start.empty()) build_buckets(ctx);
  int idx[3];
  for (int c = 0; c < 3; ++c) {
    const double t = (x[c] - ctx->bb_lo[c]) / ctx->bb_cell[c];
    if (!(t >= -1e-9 * ctx->bb_n[c]) || !(t <= ctx->bb_n[c] * (1 + 1e-9))) return false;
    idx[c] = std::min(ctx->bb_n[c] - 1, std::max(0, static_cast<int>(std::floor(t))));
  }
  const int64_t id = (static_cast<int64_t>(idx[2]) * ctx->bb_n[1] + idx[1]) * ctx->bb_n[0] + idx[0];
  for (int64_t k = ctx->bucket_start[id]; k < ctx->bucket_start[id + 1]; ++k) {
    const int64_t e = ctx->bucket_elems[k];
    const double* X = &ctx->xyz_user[12 * e];
    double J[9], Ji[9], det;
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) J[3 * r + c] = X[3 * (c + 1) + r] - X[r];
    inv3(J, Ji, &det);
    double xi[3];
    for (int r = 0; r < 3; ++r)
      xi[r] = Ji[3 * r] * (x[0] - X[0]) + Ji[3 * r + 1] * (x[1] - X[1]) + Ji[3 * r + 2] * (x[2] - X[2]);
    const double b0 = 1.0 - xi[0] - xi[1] - xi[2];
    if (b0 < -tol || xi[0] < -tol || xi[1] < -tol || xi[2] < -tol) continue;
    *elem = e;
    const double* Xs = &ctx->xyz[12 * e];
    const double* Jis = &ctx->jinv[9 * e];
    for (int r = 0; r < 3; ++r)
      xi_sorted[r] = Jis[3 * r] * (x[0] - Xs[0]) + Jis[3 * r + 1] * (x[1] - Xs[1]) + Jis[3 * r + 2] * (x[2] - Xs[2]);
    return true;
  }
  return false;
}

dg_status ensure_staging(dg_ctx* ctx, size_t bytes) {
  if (ctx->staging_bytes >= bytes) return DG_OK;
  dev_free(ctx, ctx->staging);
  ctx->staging = dev_alloc(ctx, bytes);
  ctx->staging_bytes = ctx->staging ? bytes : 0;
  if (!ctx->staging) return fail(ctx, DG_E_OOM, "staging buffer allocation failed");
  return DG_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// C-ABI
// ---------------------------------------------------------------------------

extern "C" {

int64_t dg_n_modes(int order) { return order < 0 ? 0 : n_modes(order); }

int dg_host_chunks(int64_t n_elem, int64_t* bounds, int cap) {
  if (n_elem < 1 || cap < 0 || (cap > 0 && !bounds)) return -1;
  const std::vector<int64_t> b = host_chunk_bounds(n_elem);
  const int n = static_cast<int>(b.size());
  for (int i = 0; i < n && i < cap; ++i) bounds[i] = b[static_cast<size_t>(i)];
  return n - 1;
}

const char* dg_last_error(const dg_ctx* ctx) {
  return ctx ? ctx->err.c_str() : g_last_error.c_str();
}

dg_status dg_reference_table(int order, int which, double* out, int64_t cap, int64_t* count) {
  if (!supported_order(order)) return fail(nullptr, DG_E_ORDER, "unsupported order");
  const int N = order, L = n_modes(N);
  std::vector<double> v;
  if (which == 0) {
    ref::Rule3 r = ref::volume_rule(N + 1);
    for (size_t i = 0; i < r.w.size(); ++i) v.insert(v.end(), {r.xi[i], r.eta[i], r.zeta[i], r.w[i]});
  } else if (which == 1) {
    ref::Rule2 r = ref::face_rule(N + 1);
    for (size_t i = 0; i < r.w.size(); ++i) v.insert(v.end(), {r.s[i], r.t[i], r.w[i]});
  } else if (which == 2) {
    ref::Rule1 r = ref::time_rule(N + 1);
    for (size_t i = 0; i < r.w.size(); ++i) v.insert(v.end(), {r.x[i], r.w[i]});
  } else if (which == 3 || which == 4) {
    ref::Rule3 r = ref::volume_rule(N + 1);
    std::vector<double> val(L), grd(3 * L);
    for (size_t i = 0; i < r.w.size(); ++i) {
      ref::dubiner(N, r.xi[i], r.eta[i], r.zeta[i], val.data(), grd.data());
      if (which == 3) v.insert(v.end(), val.begin(), val.end());
      else v.insert(v.end(), grd.begin(), grd.end());
    }
  } else {
    return fail(nullptr, DG_E_ARG, "unknown table");
  }
  if (count) *count = static_cast<int64_t>(v.size());
  if (out) std::memcpy(out, v.data(), sizeof(double) * std::min<int64_t>(cap, v.size()));
  return DG_OK;
}

void dg_destroy(dg_ctx* ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  while (!ctx->owned.empty()) dev_free(ctx, ctx->owned.back().first);
  if (ctx->status_host) cudaFreeHost(ctx->status_host);
  if (ctx->amp_host) cudaFreeHost(ctx->amp_host);
  for (cudaEvent_t ev : ctx->events) cudaEventDestroy(ev);
  for (cudaEvent_t ev : ctx->xfer_events) cudaEventDestroy(ev);
  if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
  delete ctx;
}

dg_status dg_mesh_create(const dg_mesh_desc* desc, dg_ctx** out) {
  if (!desc || !out) return fail(nullptr, DG_E_ARG, "NULL descriptor or output pointer");
  *out = nullptr;
  if (desc->n_elem <= 0 || !desc->elem_xyz || !desc->elem_vid)
    return fail(nullptr, DG_E_ARG, "empty mesh or NULL mesh arrays");
  if (desc->n_elem >= (int64_t(1) << 29)) return fail(nullptr, DG_E_ARG, "too many elements");
  if (!supported_order(desc->order)) return fail(nullptr, DG_E_ORDER, "order must be in 1..5");
  if (desc->members < 1) return fail(nullptr, DG_E_ARG, "members must be >= 1");
  if (!(desc->cfl > 0.0) || !std::isfinite(desc->cfl)) return fail(nullptr, DG_E_ARG, "cfl must be > 0");
  const int64_t E = desc->n_elem;
  const int64_t M = desc->members;
  if (E * M >= (int64_t(1) << 29)) return fail(nullptr, DG_E_ARG, "too many element copies (n_elem x members)");
  if (desc->face_bc)
    for (int64_t i = 0; i < 4 * E; ++i)
      if (desc->face_bc[i] < 0 || desc->face_bc[i] > 2)
        return fail(nullptr, DG_E_MESH, "face tags must be 0 (interior), 1 (free surface) or 2 (absorbing)");

  dg_ctx* ctx = new dg_ctx();
  ctx->N = desc->order;
  ctx->L = n_modes(ctx->N);
  ctx->E = E;
  ctx->M = static_cast<int>(M);
  ctx->EV = E * M;
  ctx->cfl = desc->cfl;
  ctx->stream = static_cast<cudaStream_t>(desc->cuda_stream);
  if (desc->alloc) { ctx->alloc = *desc->alloc; ctx->has_alloc = ctx->alloc.alloc && ctx->alloc.free; }

  ctx->xyz_user.assign(desc->elem_xyz, desc->elem_xyz + 12 * E);
  ctx->xyz.resize(12 * E);
  ctx->jinv.resize(9 * E);
  ctx->detj.resize(E);
  ctx->rin.resize(E);
  std::vector<int64_t> vid_sorted(4 * E);
  std::vector<int8_t> bc_sorted(4 * E, 0);
  std::vector<GeomF> geom(E);
  for (int64_t e = 0; e < E; ++e) {
    const int64_t* v = desc->elem_vid + 4 * e;
    std::array<int, 4> ord{0, 1, 2, 3};
    std::sort(ord.begin(), ord.end(), [&](int a, int b) { return v[a] < v[b]; });
    for (int j = 0; j < 3; ++j)
      if (v[ord[j]] == v[ord[j + 1]]) { dg_destroy(ctx); return fail(nullptr, DG_E_MESH, "element " + std::to_string(e) + " repeats a vertex id"); }
    for (int j = 0; j < 4; ++j) {
      vid_sorted[4 * e + j] = v[ord[j]];
      if (desc->face_bc) bc_sorted[4 * e + j] = desc->face_bc[4 * e + ord[j]];   // face j is opposite vertex j
      for (int c = 0; c < 3; ++c) ctx->xyz[12 * e + 3 * j + c] = desc->elem_xyz[12 * e + 3 * ord[j] + c];
    }
    const double* X = &ctx->xyz[12 * e];
    double J[9], det;
    double scale = 0.0;
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) {
        J[3 * r + c] = X[3 * (c + 1) + r] - X[r];
        scale = std::max(scale, std::fabs(J[3 * r + c]));
      }
    double* Ji = &ctx->jinv[9 * e];
    inv3(J, Ji, &det);
    if (!std::isfinite(det) || std::fabs(det) <= 1e-12 * scale * scale * scale) {
      dg_destroy(ctx);
      return fail(nullptr, DG_E_MESH, "element " + std::to_string(e) + " is degenerate");
    }
    ctx->detj[e] = std::fabs(det);
    GeomF& g = geom[e];
    std::memset(&g, 0, sizeof(g));
    for (int k = 0; k < 9; ++k) g.tinv[k] = static_cast<float>(Ji[k]);
    g.inv_detj = static_cast<float>(1.0 / ctx->detj[e]);
    double area_sum = 0.0;
    for (int f = 0; f < 4; ++f) {
      int a[3], n = 0;
      for (int j = 0; j < 4; ++j) if (j != f) a[n++] = j;
      const double* A = X + 3 * a[0];
      const double* B = X + 3 * a[1];
      const double* C = X + 3 * a[2];
      const double u[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
      const double w[3] = {C[0] - A[0], C[1] - A[1], C[2] - A[2]};
      double nrm[3] = {u[1] * w[2] - u[2] * w[1], u[2] * w[0] - u[0] * w[2], u[0] * w[1] - u[1] * w[0]};
      const double len = std::sqrt(nrm[0] * nrm[0] + nrm[1] * nrm[1] + nrm[2] * nrm[2]);
      const double* P = X + 3 * f;
      const double side = nrm[0] * (P[0] - A[0]) + nrm[1] * (P[1] - A[1]) + nrm[2] * (P[2] - A[2]);
      const double sgn = side > 0 ? -1.0 : 1.0;
      for (int c = 0; c < 3; ++c) g.face[f][c] = static_cast<float>(sgn * nrm[c] / len);
      g.face[f][3] = static_cast<float>(0.5 * len / ctx->detj[e]);
      area_sum += 0.5 * len;
    }
    ctx->rin[e] = 3.0 * (ctx->detj[e] / 6.0) / area_sum;
  }

  // face matching by vertex-id triples (ascending in the sorted order); a tagged
  // boundary face must belong to one element only (map value kBoundary)
  std::vector<int> nbr(4 * E, -1);
  {
    constexpr int64_t kMatched = -1, kBoundary = -2;
    std::unordered_map<FaceKey, int64_t, FaceKeyHash> open;
    open.reserve(static_cast<size_t>(2 * E + 16));
    for (int64_t e = 0; e < E; ++e)
      for (int f = 0; f < 4; ++f) {
        int a[3], n = 0;
        for (int j = 0; j < 4; ++j) if (j != f) a[n++] = j;
        FaceKey key{vid_sorted[4 * e + a[0]], vid_sorted[4 * e + a[1]], vid_sorted[4 * e + a[2]]};
        const bool tagged = bc_sorted[4 * e + f] != 0;
        auto it = open.find(key);
        if (it == open.end()) {
          open.emplace(key, tagged ? kBoundary : 4 * e + f);
        } else {
          const int64_t other = it->second;
          if (tagged || other == kBoundary) {
            dg_destroy(ctx);
            return fail(nullptr, DG_E_MESH, "boundary face of element " + std::to_string(e) + " is shared with another element");
          }
          if (other == kMatched || other / 4 == e) {
            dg_destroy(ctx);
            return fail(nullptr, DG_E_MESH, "face of element " + std::to_string(e) + " is shared more than twice or with itself");
          }
          nbr[4 * e + f] = static_cast<int>(other);                       // (elem << 2) | face
          nbr[other] = static_cast<int>(4 * e + f);
          it->second = kMatched;
        }
      }
    for (const auto& kv : open)
      if (kv.second >= 0) {
        dg_destroy(ctx);
        return fail(nullptr, DG_E_MESH, "unmatched interior face of element " + std::to_string(kv.second / 4));
      }
  }

  // face list: each interior face once, first seen from its lower-index element;
  // then the boundary faces as (element, face, -1, tag)
  std::vector<int4> faces;
  std::vector<int> elem_face(4 * E, -1);
  faces.reserve(static_cast<size_t>(2 * E));
  for (int64_t e = 0; e < E; ++e)
    for (int f = 0; f < 4; ++f) {
      if (elem_face[4 * e + f] >= 0 || bc_sorted[4 * e + f] != 0) continue;
      const int other = nbr[4 * e + f];
      const int64_t fid = static_cast<int64_t>(faces.size());
      faces.push_back(make_int4(static_cast<int>(e), f, other >> 2, other & 3));
      elem_face[4 * e + f] = static_cast<int>(fid << 1);
      elem_face[other] = static_cast<int>((fid << 1) | 1);
    }
  ctx->F_interior = static_cast<int64_t>(faces.size());
  for (int64_t e = 0; e < E; ++e)
    for (int f = 0; f < 4; ++f)
      if (bc_sorted[4 * e + f] != 0) {
        elem_face[4 * e + f] = static_cast<int>(static_cast<int64_t>(faces.size()) << 1);
        faces.push_back(make_int4(static_cast<int>(e), f, -1, bc_sorted[4 * e + f]));
      }
  ctx->F = static_cast<int64_t>(faces.size());
  if (ctx->F * M >= (int64_t(1) << 30)) {
    dg_destroy(ctx);
    return fail(nullptr, DG_E_ARG, "too many faces x members");
  }
  if (M == 1) {
    // the face ranges that dg_step_host launches as soon as their predictors are done
    const std::vector<int64_t> cb = host_chunk_bounds(E);
    const int C = static_cast<int>(cb.size()) - 1;
    ctx->host_faces.assign(static_cast<size_t>(C), HostChunkFaces{});
    int64_t fi = 0, fb = ctx->F_interior;
    for (int k = 0; k < C; ++k) {
      const int64_t e1 = cb[static_cast<size_t>(k) + 1];
      HostChunkFaces& h = ctx->host_faces[static_cast<size_t>(k)];
      int64_t reach = cb[static_cast<size_t>(k)];
      h.fi0 = fi;
      for (; fi < ctx->F_interior && faces[static_cast<size_t>(fi)].x < e1; ++fi)
        reach = std::max<int64_t>(reach, faces[static_cast<size_t>(fi)].z);
      h.fi1 = fi;
      h.need = host_chunk_of(cb, reach);
      h.fb0 = fb;
      for (; fb < ctx->F && faces[static_cast<size_t>(fb)].x < e1; ++fb) {}
      h.fb1 = fb;
    }
  }

  // ensemble: copy v = e * M + m of element e for member m, and copy fid * M + m of face fid;
  // member m's copies only see each other
  if (M > 1) {
    const int64_t EV = E * M;
    std::vector<GeomF> geom_v(EV);
    std::vector<int> nbr_v(4 * EV, -1), elem_face_v(4 * EV, -1);
    std::vector<int4> faces_v(ctx->F * M);
    for (int64_t e = 0; e < E; ++e)
      for (int64_t m = 0; m < M; ++m) {
        const int64_t v = e * M + m;
        geom_v[v] = geom[e];
        for (int f = 0; f < 4; ++f) {
          const int nb = nbr[4 * e + f];
          if (nb >= 0) nbr_v[4 * v + f] = static_cast<int>((((nb >> 2) * M + m) << 2) | (nb & 3));
          const int ef = elem_face[4 * e + f];
          elem_face_v[4 * v + f] = static_cast<int>((((ef >> 1) * M + m) << 1) | (ef & 1));
        }
      }
    for (int64_t fid = 0; fid < ctx->F; ++fid)
      for (int64_t m = 0; m < M; ++m) {
        const int4 fa = faces[fid];
        faces_v[fid * M + m] = make_int4(static_cast<int>(fa.x * M + m), fa.y,
                                         fa.z < 0 ? fa.z : static_cast<int>(fa.z * M + m), fa.w);
      }
    geom.swap(geom_v);
    nbr.swap(nbr_v);
    elem_face.swap(elem_face_v);
    faces.swap(faces_v);
    ctx->F *= M;
    ctx->F_interior *= M;
  }

  // device allocation and upload
  const int N = ctx->N;
  const size_t qs = static_cast<size_t>(q_stride(N)), ds = static_cast<size_t>(d_stride(N));
  const int64_t EV = ctx->EV;
  ctx->q[0] = static_cast<float*>(dev_alloc(ctx, sizeof(float) * qs * EV));
  ctx->q[1] = static_cast<float*>(dev_alloc(ctx, sizeof(float) * qs * EV));
  ctx->d = static_cast<float*>(dev_alloc(ctx, sizeof(float) * ds * EV));
  ctx->cp = static_cast<float*>(dev_alloc(ctx, sizeof(float) * EV));
  ctx->ff = static_cast<float*>(dev_alloc(ctx, sizeof(float) * ff_stride(N) * ctx->F));
  ctx->faces = static_cast<int4*>(dev_alloc(ctx, sizeof(int4) * ctx->F));
  ctx->elem_face = static_cast<int*>(dev_alloc(ctx, sizeof(int) * 4 * EV));
  ctx->geom = static_cast<GeomF*>(dev_alloc(ctx, sizeof(GeomF) * EV));
  ctx->matf = static_cast<MatF*>(dev_alloc(ctx, sizeof(MatF) * EV));
  ctx->nbr = static_cast<int*>(dev_alloc(ctx, sizeof(int) * 4 * EV));
  const TableLayout TL = table_layout(N);
  ctx->tables = static_cast<float*>(dev_alloc(ctx, sizeof(float) * TL.total));
  ctx->status = static_cast<unsigned*>(dev_alloc(ctx, sizeof(unsigned)));
  if (!ctx->q[0] || !ctx->q[1] || !ctx->d || !ctx->cp || !ctx->ff || !ctx->faces || !ctx->elem_face ||
      !ctx->geom || !ctx->matf || !ctx->nbr ||
      !ctx->tables || !ctx->status) {
    dg_destroy(ctx);
    return fail(nullptr, DG_E_OOM, "device allocation failed");
  }
  if (cudaMallocHost(&ctx->status_host, sizeof(unsigned)) != cudaSuccess) {
    cudaGetLastError();
    dg_destroy(ctx);
    return fail(nullptr, DG_E_OOM, "pinned allocation failed");
  }
  std::vector<float> tf;
  {
    std::vector<double> t = build_tables(N);
    tf.assign(t.begin(), t.end());
  }
  dg_status st;
  if ((st = upload(ctx, ctx->geom, geom.data(), sizeof(GeomF) * EV)) != DG_OK ||
      (st = upload(ctx, ctx->nbr, nbr.data(), sizeof(int) * 4 * EV)) != DG_OK ||
      (st = upload(ctx, ctx->faces, faces.data(), sizeof(int4) * ctx->F)) != DG_OK ||
      (st = upload(ctx, ctx->elem_face, elem_face.data(), sizeof(int) * 4 * EV)) != DG_OK ||
      (st = upload(ctx, ctx->tables, tf.data(), sizeof(float) * tf.size())) != DG_OK) {
    std::string m = ctx->err;
    dg_destroy(ctx);
    return fail(nullptr, st, m);
  }
  cudaError_t ce;
  if ((ce = cudaMemsetAsync(ctx->q[0], 0, sizeof(float) * qs * EV, ctx->stream)) != cudaSuccess ||
      (ce = cudaMemsetAsync(ctx->q[1], 0, sizeof(float) * qs * EV, ctx->stream)) != cudaSuccess ||
      (ce = cudaMemsetAsync(ctx->d, 0, sizeof(float) * ds * EV, ctx->stream)) != cudaSuccess ||
      (ce = cudaStreamSynchronize(ctx->stream)) != cudaSuccess) {
    dg_destroy(ctx);
    return fail(nullptr, DG_E_CUDA, std::string("initialising device memory: ") + cudaGetErrorString(ce));
  }
  {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sms > 0) {
      ctx->grid_pred = ctx->grid_face = ctx->grid_corr = sms;
    }
    cudaGetLastError();
  }
  *out = ctx;
  return DG_OK;
}

dg_status dg_set_predictor(dg_ctx* ctx, int kind, int iterations) {
  if (!ctx) return fail(ctx, DG_E_ARG, "NULL context");
  if (kind == DG_PREDICTOR_CK) {
    ctx->picard_iters = 0;
    return DG_OK;
  }
  if (kind != DG_PREDICTOR_PICARD || iterations < 1 || iterations > 16)
    return fail(ctx, DG_E_ARG, "unknown predictor or iteration count");
  if (ctx->N > 4) return fail(ctx, DG_E_ORDER, "the Picard predictor supports degrees 1..4");
  ctx->picard_iters = iterations;
  return DG_OK;
}

dg_status dg_set_wait_limit(dg_ctx* ctx, int64_t polls) {
  if (!ctx) return fail(ctx, DG_E_ARG, "NULL context");
  if (polls > INT32_MAX) return fail(ctx, DG_E_ARG, "wait limit above 2^31 - 1 polls");
  ctx->wait_limit = polls < 0 ? -1 : static_cast<int>(polls);
  return DG_OK;
}

dg_status dg_set_rheology(dg_ctx* ctx, int law) {
  if (!ctx) return fail(ctx, DG_E_ARG, "NULL context");
  if (law != DG_LAW_CDM && law != DG_LAW_IVM && law != DG_LAW_NLSHEAR) return fail(ctx, DG_E_ARG, "unknown rheology");
  if (law != ctx->law) ctx->has_material = false;   // the material slots change meaning
  ctx->law = law;
  return DG_OK;
}

dg_status dg_set_material(dg_ctx* ctx, const double* mat, const double* member_xi0_cd) {
  if (!ctx || !mat) return fail(ctx, DG_E_ARG, "NULL argument");
  if (member_xi0_cd && ctx->M == 1) return fail(ctx, DG_E_ARG, "per-member parameters need members > 1");
  if (member_xi0_cd && ctx->law != DG_LAW_CDM) return fail(ctx, DG_E_ARG, "per-member parameters are CDM (xi0, C_d)");
  const int64_t E = ctx->E, M = ctx->M;
  std::vector<MatF> mf(ctx->EV);
  double dt = INFINITY;
  for (int64_t e = 0; e < E; ++e) {
    const double* m = mat + 6 * e;
    for (int k = 0; k < 6; ++k)
      if (!std::isfinite(m[k])) return fail(ctx, DG_E_ARG, "non-finite material of element " + std::to_string(e));
    const double rho = m[0], lam = m[1], mu = m[2], gr = m[3];
    if (!(rho > 0) || !(mu > 0) || !(lam + 2 * mu > 0))
      return fail(ctx, DG_E_ARG, "invalid material of element " + std::to_string(e));
    if (ctx->law == DG_LAW_NLSHEAR) {
      // (rho, lambda0, mu0, beta, -, -): beta in gamma_r
      if (!(m[3] >= 0)) return fail(ctx, DG_E_ARG, "the shear law needs beta >= 0, element " + std::to_string(e));
      const MatF f{float(rho), float(lam), float(mu), float(m[3]), 0.f, 0.f, float(1.0 / rho), 0.f};
      for (int64_t k = 0; k < M; ++k) mf[e * M + k] = f;
      const double cp = std::sqrt((lam + 2 * mu) / rho);
      dt = std::min(dt, ctx->cfl * 2.0 * ctx->rin[e] / ((2 * ctx->N + 1) * cp));
      continue;
    }
    if (ctx->law == DG_LAW_IVM) {
      // (rho, lambda0, mu0, gamma_b, tau_b, -): gamma_b in gamma_r, 1/(gamma_b tau_b) in C_d
      if (!(m[3] > 0) || !(m[4] > 0)) return fail(ctx, DG_E_ARG, "IVM needs gamma_b > 0 and tau_b > 0, element " + std::to_string(e));
      const MatF f{float(rho), float(lam), float(mu), float(m[3]), float(m[4]), float(1.0 / (m[3] * m[4])),
                   float(1.0 / rho), 0.f};
      for (int64_t k = 0; k < M; ++k) mf[e * M + k] = f;
      const double cp = std::sqrt((lam + 2 * mu) / rho);
      dt = std::min(dt, ctx->cfl * 2.0 * ctx->rin[e] / ((2 * ctx->N + 1) * cp));
      continue;
    }
    if (gr < 0 || m[5] < 0) return fail(ctx, DG_E_ARG, "invalid material of element " + std::to_string(e));
    for (int64_t k = 0; k < M; ++k) {
      double xi0 = m[4], cd = m[5];
      if (member_xi0_cd) {
        xi0 = member_xi0_cd[2 * (k * E + e)];
        cd = member_xi0_cd[2 * (k * E + e) + 1];
        if (!std::isfinite(xi0) || !std::isfinite(cd) || cd < 0)
          return fail(ctx, DG_E_ARG, "invalid member parameters of element " + std::to_string(e));
      }
      mf[e * M + k] = MatF{float(rho), float(lam), float(mu), float(gr), float(xi0), float(cd), float(1.0 / rho), 0.f};
    }
    const double cp = std::sqrt((lam + 2 * mu) / rho);
    dt = std::min(dt, ctx->cfl * 2.0 * ctx->rin[e] / ((2 * ctx->N + 1) * cp));
  }
  ctx->mat.assign(mat, mat + 6 * E);
  dg_status st = upload(ctx, ctx->matf, mf.data(), sizeof(MatF) * ctx->EV);
  if (st != DG_OK) return st;
  ctx->dt_cfl = dt;
  ctx->has_material = true;
  return DG_OK;
}

double dg_dt(const dg_ctx* ctx) { return ctx ? ctx->dt_cfl : 0.0; }
double dg_time(const dg_ctx* ctx) { return ctx ? ctx->t : 0.0; }

dg_status dg_get_stats(const dg_ctx* ctx, dg_stats* out) {
  if (!ctx || !out) return fail(const_cast<dg_ctx*>(ctx), DG_E_ARG, "NULL argument");
  *out = ctx->stats;
  return DG_OK;
}

static dg_status set_state_impl(dg_ctx* ctx, const void* q, int is_double, bool device, double t) {
  if (!ctx || !q) return fail(ctx, DG_E_ARG, "NULL argument");
  if (!std::isfinite(t)) return fail(ctx, DG_E_ARG, "non-finite time");
  const size_t n = static_cast<size_t>(ctx->EV) * kFields * ctx->L;
  const void* src = q;
  if (!device) {
    dg_status st = ensure_staging(ctx, n * (is_double ? 8 : 4));
    if (st != DG_OK) return st;
    DG_CUDA(ctx, cudaMemcpyAsync(ctx->staging, q, n * (is_double ? 8 : 4), cudaMemcpyHostToDevice, ctx->stream));
    src = ctx->staging;
  }
  DG_CUDA(ctx, launch_state_in(ctx->N, ctx->E, ctx->M, src, is_double, ctx->q[ctx->cur], ctx->stream));
  if (!device) DG_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  ctx->t = t;
  ctx->has_state = true;
  return DG_OK;
}

dg_status dg_set_state(dg_ctx* ctx, const double* q, double t) { return set_state_impl(ctx, q, 1, false, t); }
dg_status dg_set_state_f32(dg_ctx* ctx, const float* q, double t) { return set_state_impl(ctx, q, 0, false, t); }
dg_status dg_set_state_device(dg_ctx* ctx, const float* q, double t) { return set_state_impl(ctx, q, 0, true, t); }

static dg_status get_state_impl(dg_ctx* ctx, void* q, int is_double, bool device, double* t_out) {
  if (!ctx || !q) return fail(ctx, DG_E_ARG, "NULL argument");
  const size_t n = static_cast<size_t>(ctx->EV) * kFields * ctx->L;
  void* dst = q;
  if (!device) {
    dg_status st = ensure_staging(ctx, n * (is_double ? 8 : 4));
    if (st != DG_OK) return st;
    dst = ctx->staging;
  }
  DG_CUDA(ctx, launch_state_out(ctx->N, ctx->E, ctx->M, ctx->q[ctx->cur], dst, is_double, ctx->stream));
  if (!device) DG_CUDA(ctx, cudaMemcpyAsync(q, ctx->staging, n * (is_double ? 8 : 4), cudaMemcpyDeviceToHost, ctx->stream));
  DG_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (t_out) *t_out = ctx->t;
  return DG_OK;
}

dg_status dg_get_state(dg_ctx* ctx, double* q, double* t) { return get_state_impl(ctx, q, 1, false, t); }
dg_status dg_get_state_f32(dg_ctx* ctx, float* q, double* t) { return get_state_impl(ctx, q, 0, false, t); }
dg_status dg_get_state_device(dg_ctx* ctx, float* q, double* t) { return get_state_impl(ctx, q, 0, true, t); }

dg_status dg_set_source(dg_ctx* ctx, const dg_point_source* src, int64_t n) {
  if (!ctx || n < 0 || (n > 0 && !src)) return fail(ctx, DG_E_ARG, "invalid source list");
  if (!ctx->has_material) return fail(ctx, DG_E_STATE, "dg_set_material must precede dg_set_source");
  if (ctx->L > 64) return fail(ctx, DG_E_ORDER, "order too high for point sources");
  const int64_t M = ctx->M;
  std::vector<SourceDev> host(n * M);
  std::vector<double> phi(ctx->L);
  for (int64_t s = 0; s < n; ++s) {
    const dg_point_source& p = src[s];
    if (p.stf != 0 && p.stf != 1) return fail(ctx, DG_E_ARG, "unknown source time function");
    if (!(p.f0_or_sigma > 0)) return fail(ctx, DG_E_ARG, "source f0/sigma must be > 0");
    int64_t e;
    double xi[3];
    if (!locate(ctx, p.x, &e, xi)) return fail(ctx, DG_E_OUTSIDE, "source " + std::to_string(s) + " lies outside the mesh");
    ref::dubiner(ctx->N, xi[0], xi[1], xi[2], phi.data(), nullptr);
    const double lam = ctx->mat[6 * e + 1], mu = ctx->mat[6 * e + 2];
    const double tr = p.m[0] + p.m[1] + p.m[2];
    double eps[6];
    for (int k = 0; k < 6; ++k) eps[k] = p.m[k] / (2.0 * mu);
    for (int k = 0; k < 3; ++k) eps[k] -= lam / (2.0 * mu * (3.0 * lam + 2.0 * mu)) * tr;
    SourceDev& d = host[s * M];
    std::memset(&d, 0, sizeof(d));
    d.elem = e * M;
    for (int k = 0; k < 6; ++k)
      for (int l = 0; l < ctx->L; ++l) d.phi_eps[k * ctx->L + l] = static_cast<float>(phi[l] * eps[k] / ctx->detj[e]);
    for (int64_t m = 1; m < M; ++m) {            // the same source in every member
      host[s * M + m] = d;
      host[s * M + m].elem = e * M + m;
    }
  }
  dev_free(ctx, ctx->source_dev);
  ctx->source_dev = nullptr;
  ctx->sources.assign(src, src + n);
  ctx->source_host = host;
  if (n > 0) {
    ctx->source_dev = static_cast<SourceDev*>(dev_alloc(ctx, sizeof(SourceDev) * n * M));
    if (!ctx->source_dev) return fail(ctx, DG_E_OOM, "source allocation failed");
    return upload(ctx, ctx->source_dev, host.data(), sizeof(SourceDev) * n * M);
  }
  return DG_OK;
}

dg_status dg_receivers(dg_ctx* ctx, const double* xyz, int64_t R) {
  if (!ctx || R < 0 || (R > 0 && !xyz)) return fail(ctx, DG_E_ARG, "invalid receiver list");
  if (ctx->L > 64) return fail(ctx, DG_E_ORDER, "order too high for receivers");
  const int64_t M = ctx->M;
  std::vector<ReceiverDev> host(R * M);
  std::vector<double> phi(ctx->L);
  for (int64_t r = 0; r < R; ++r) {
    int64_t e;
    double xi[3];
    if (!locate(ctx, xyz + 3 * r, &e, xi)) return fail(ctx, DG_E_OUTSIDE, "receiver " + std::to_string(r) + " lies outside the mesh");
    ref::dubiner(ctx->N, xi[0], xi[1], xi[2], phi.data(), nullptr);
    for (int64_t m = 0; m < M; ++m) {           // member m's copy of receiver r at m * R + r
      ReceiverDev& h = host[m * R + r];
      std::memset(&h, 0, sizeof(ReceiverDev));
      h.elem = e * M + m;
      for (int l = 0; l < ctx->L; ++l) h.phi[l] = static_cast<float>(phi[l]);
    }
  }
  dev_free(ctx, ctx->rec_dev);
  dev_free(ctx, ctx->traces);
  ctx->rec_dev = nullptr;
  ctx->traces = nullptr;
  ctx->trace_cap = 0;
  ctx->n_rec = 0;
  ctx->rec_host = host;
  if (R > 0) {
    ctx->rec_dev = static_cast<ReceiverDev*>(dev_alloc(ctx, sizeof(ReceiverDev) * R * M));
    if (!ctx->rec_dev) return fail(ctx, DG_E_OOM, "receiver allocation failed");
    return upload(ctx, ctx->rec_dev, host.data(), sizeof(ReceiverDev) * R * M);
  }
  return DG_OK;
}

dg_status dg_receivers_read(dg_ctx* ctx, float* out, int64_t cap, int64_t* n_rec) {
  if (!ctx) return fail(ctx, DG_E_ARG, "NULL context");
  const int64_t R = static_cast<int64_t>(ctx->rec_host.size());
  if (n_rec) *n_rec = ctx->n_rec;
  const int64_t n = std::min(cap, ctx->n_rec);
  if (n > 0 && R > 0) {
    if (!out) return fail(ctx, DG_E_ARG, "NULL output");
    DG_CUDA(ctx, cudaMemcpyAsync(out, ctx->traces, sizeof(float) * 3 * R * n, cudaMemcpyDeviceToHost, ctx->stream));
  }
  DG_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return DG_OK;
}

dg_status dg_profile_enable(dg_ctx* ctx, int on) {
  if (!ctx) return fail(ctx, DG_E_ARG, "NULL context");
  ctx->profiling = on != 0;
  std::memset(ctx->prof, 0, sizeof(ctx->prof));
  return DG_OK;
}

dg_status dg_profile_read(dg_ctx* ctx, dg_kernel_time* out, int cap, int* n_kinds) {
  if (!ctx) return fail(ctx, DG_E_ARG, "NULL context");
  if (n_kinds) *n_kinds = 5;
  for (int k = 0; k < std::min(cap, 5); ++k) out[k] = ctx->prof[k];
  return DG_OK;
}

static double stf_integral(const dg_point_source& s, double t) {
  const double tau = t - s.t0;
  if (s.stf == 0) {
    const double c = (M_PI * s.f0_or_sigma) * (M_PI * s.f0_or_sigma);
    return tau * std::exp(-c * tau * tau);
  }
  return 0.5 * (1.0 + std::erf(tau / (s.f0_or_sigma * std::sqrt(2.0))));
}

namespace {

// Per-call preparation of a run of n_steps steps of size dt: the sources' amplitude
// per step (exact time integrals of the moment-rate function) and room for the
// receivers' traces.
dg_status prepare_steps(dg_ctx* ctx, int64_t n_steps, double dt) {
  const int nsrc = static_cast<int>(ctx->source_host.size());     // sources x members
  const int R = static_cast<int>(ctx->rec_host.size());           // receivers x members
  const int M = ctx->M;
  // per-step source amplitudes (exact time integrals of the moment-rate function)
  if (nsrc > 0) {
    const int64_t need = n_steps * nsrc;
    if (ctx->amp_cap < need) {
      dev_free(ctx, ctx->amp_dev);
      if (ctx->amp_host) cudaFreeHost(ctx->amp_host);
      ctx->amp_host = nullptr;
      ctx->amp_dev = static_cast<float*>(dev_alloc(ctx, sizeof(float) * need));
      if (!ctx->amp_dev || cudaMallocHost(&ctx->amp_host, sizeof(float) * need) != cudaSuccess) {
        ctx->amp_cap = 0;
        return fail(ctx, DG_E_OOM, "source amplitude buffer");
      }
      ctx->amp_cap = need;
    }
    DG_CUDA(ctx, cudaStreamSynchronize(ctx->stream));     // amp_host may still be read by a copy
    for (int64_t s = 0; s < n_steps; ++s) {
      const double t0 = ctx->t + s * dt, t1 = ctx->t + (s + 1) * dt;
      for (int k = 0; k < nsrc; ++k)
        ctx->amp_host[s * nsrc + k] =
            static_cast<float>(stf_integral(ctx->sources[k / M], t1) - stf_integral(ctx->sources[k / M], t0));
    }
    DG_CUDA(ctx, cudaMemcpyAsync(ctx->amp_dev, ctx->amp_host, sizeof(float) * need, cudaMemcpyHostToDevice, ctx->stream));
  }
  // receiver trace capacity
  if (R > 0) {
    const int64_t need = std::min<int64_t>(ctx->n_rec + n_steps, 65536);
    if (need > ctx->trace_cap) {
      int64_t cap = std::max<int64_t>(1024, ctx->trace_cap);
      while (cap < need) cap *= 2;
      cap = std::min<int64_t>(cap, 65536);
      float* nt = static_cast<float*>(dev_alloc(ctx, sizeof(float) * 3 * R * cap));
      if (!nt) return fail(ctx, DG_E_OOM, "trace buffer");
      if (ctx->traces && ctx->n_rec > 0)
        DG_CUDA(ctx, cudaMemcpyAsync(nt, ctx->traces, sizeof(float) * 3 * R * ctx->n_rec, cudaMemcpyDeviceToDevice, ctx->stream));
      dev_free(ctx, ctx->traces);
      ctx->traces = nt;
      ctx->trace_cap = cap;
    }
  }
  return DG_OK;
}

}  // namespace

dg_status dg_step(dg_ctx* ctx, int64_t n_steps, double dt) {
  if (!ctx) return fail(ctx, DG_E_ARG, "NULL context");
  if (n_steps < 0) return fail(ctx, DG_E_ARG, "negative step count");
  if (!ctx->has_material || !ctx->has_state) return fail(ctx, DG_E_STATE, "material and state must be set before dg_step");
  if (dt <= 0) dt = ctx->dt_cfl;
  if (!std::isfinite(dt)) return fail(ctx, DG_E_ARG, "non-finite dt");
  if (n_steps == 0) return DG_OK;
  const int nsrc = static_cast<int>(ctx->source_host.size());     // sources x members
  const int R = static_cast<int>(ctx->rec_host.size());           // receivers x members
  {
    dg_status st = prepare_steps(ctx, n_steps, dt);
    if (st != DG_OK) return st;
  }
  DG_CUDA(ctx, cudaMemsetAsync(ctx->status, 0, sizeof(unsigned), ctx->stream));
  // events for per-kernel timing
  const int per_step = 3 + (nsrc > 0) + (R > 0);
  if (ctx->profiling) {
    const size_t need = static_cast<size_t>(n_steps * per_step + 1);
    while (ctx->events.size() < need) {
      cudaEvent_t ev;
      DG_CUDA(ctx, cudaEventCreate(&ev));
      ctx->events.push_back(ev);
    }
    ctx->event_kind.assign(need, -1);
  }
  size_t ev = 0;
  auto mark = [&](int kind) -> cudaError_t {
    if (!ctx->profiling) return cudaSuccess;
    if (kind >= 0) ctx->event_kind[ev] = kind;
    return cudaEventRecord(ctx->events[ev++], ctx->stream);
  };
  StepArgs a{};
  a.E = ctx->EV;
  a.F = ctx->F;
  a.has_boundary = ctx->F > ctx->F_interior;
  a.d = ctx->d;
  a.cp = ctx->cp;
  a.ff = ctx->ff;
  a.faces = ctx->faces;
  a.elem_face = ctx->elem_face;
  a.grid_pred = ctx->grid_pred;
  a.grid_face = ctx->grid_face;
  a.grid_corr = ctx->grid_corr;
  a.law = ctx->law;
  a.picard_iters = ctx->picard_iters;
  a.wait_limit = ctx->wait_limit;
  a.wait_limit_set = ctx->wait_limit >= 0;
  a.geom = ctx->geom;
  a.mat = ctx->matf;
  a.nbr = ctx->nbr;
  a.tables = ctx->tables;
  a.dt = static_cast<float>(dt);
  a.status = ctx->status;
  int64_t launches = 0;
  DG_CUDA(ctx, mark(-1));
  for (int64_t s = 0; s < n_steps; ++s) {
    a.q_in = ctx->q[ctx->cur];
    a.q_out = ctx->q[1 - ctx->cur];
    DG_CUDA(ctx, launch_predictor(ctx->N, a, ctx->stream));
    if (a.picard_iters > 0) {
      DG_CUDA(ctx, launch_picard(ctx->N, a, ctx->stream));
      ++launches;
    }
    DG_CUDA(ctx, mark(0));
    DG_CUDA(ctx, launch_faces(ctx->N, a, ctx->stream));
    DG_CUDA(ctx, mark(4));
    DG_CUDA(ctx, launch_corrector(ctx->N, a, ctx->stream));
    DG_CUDA(ctx, mark(1));
    launches += 3;
    ctx->cur = 1 - ctx->cur;
    if (nsrc > 0) {
      DG_CUDA(ctx, launch_sources(ctx->N, nsrc, ctx->source_dev, ctx->amp_dev, s, ctx->q[ctx->cur], ctx->stream));
      DG_CUDA(ctx, mark(2));
      ++launches;
    }
    if (R > 0) {
      if (ctx->n_rec < 65536) {
        DG_CUDA(ctx, launch_receivers(ctx->N, R, ctx->rec_dev, ctx->q[ctx->cur], ctx->traces + 3 * R * ctx->n_rec, ctx->stream));
        ++ctx->n_rec;
        ++launches;
      }
      DG_CUDA(ctx, mark(3));
    }
  }
  DG_CUDA(ctx, cudaMemcpyAsync(ctx->status_host, ctx->status, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->stream));
  DG_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  ctx->t += n_steps * dt;
  ctx->stats.steps += n_steps;
  ctx->stats.kernel_launches += launches;
  ctx->stats.element_updates += n_steps * ctx->EV;
  if (ctx->profiling) {
    for (size_t i = 1; i < ev; ++i) {
      float ms = 0.f;
      DG_CUDA(ctx, cudaEventElapsedTime(&ms, ctx->events[i - 1], ctx->events[i]));
      const int k = ctx->event_kind[i];
      if (k >= 0 && k < 5) {
        ctx->prof[k].launches += 1;
        ctx->prof[k].total_ms += ms;
      }
    }
  }
  const unsigned st = *ctx->status_host;
  if (st & kStatusNonFinite) return fail(ctx, DG_E_NONFINITE, "non-finite value in the state");
  if (st & kStatusNonHyperbolic) return fail(ctx, DG_E_NONHYPERBOLIC, "effective moduli lost hyperbolicity");
  if (st & kStatusIndex) return fail(ctx, DG_E_MESH, "neighbour index out of range");
  if (st & kStatusTimeout) return fail(ctx, DG_E_CUDA, "a bounded wait on the tensor cores timed out");
  return DG_OK;
}

// One step from a host state to a host state, with the transfers overlapped: the
// element range is cut into chunks (host_chunk_bounds); the host-to-device copy of
// chunk k+1 runs (on a copy stream) while chunk k is converted and predicted, the
// faces run as soon as their two sides are predicted, and the device-to-host copy of
// chunk k runs while the corrector works on chunk k+1.  Every element's arithmetic
// is the same as dg_step's.
dg_status dg_step_host(dg_ctx* ctx, const float* q_in, float* q_out, double dt) {
  if (!ctx || !q_in || !q_out) return fail(ctx, DG_E_ARG, "NULL argument");
  if (!ctx->has_material) return fail(ctx, DG_E_STATE, "material must be set before dg_step_host");
  if (ctx->M != 1) {                        // members: the plain sequence
    dg_status st = dg_set_state_f32(ctx, q_in, ctx->t);
    if (st == DG_OK) st = dg_step(ctx, 1, dt);
    double t = 0.0;
    return st == DG_OK ? dg_get_state_f32(ctx, q_out, &t) : st;
  }
  if (dt <= 0) dt = ctx->dt_cfl;
  if (!std::isfinite(dt)) return fail(ctx, DG_E_ARG, "non-finite dt");
  const int nsrc = static_cast<int>(ctx->source_host.size());
  const int R = static_cast<int>(ctx->rec_host.size());
  {
    dg_status st = prepare_steps(ctx, 1, dt);
    if (st != DG_OK) return st;
  }
  const int64_t E = ctx->E, L = ctx->L;
  const size_t row = static_cast<size_t>(kFields * L);          // floats per element, host layout
  const int64_t qs = q_stride(ctx->N), ds = d_stride(ctx->N);
  {
    dg_status st = ensure_staging(ctx, sizeof(float) * row * E);
    if (st != DG_OK) return st;
  }
  const std::vector<int64_t> cb = host_chunk_bounds(E);
  const int C = static_cast<int>(cb.size()) - 1;
  const bool face_ranges = ctx->host_faces.size() == static_cast<size_t>(C);
  if (!ctx->copy_stream) DG_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
  while (ctx->xfer_events.size() < static_cast<size_t>(2 * C + 1)) {
    cudaEvent_t ev;
    DG_CUDA(ctx, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    ctx->xfer_events.push_back(ev);
  }
  cudaEvent_t* evH = ctx->xfer_events.data();
  cudaEvent_t* evC = evH + C;
  cudaEvent_t evStart = evH[2 * C];
  float* staging = static_cast<float*>(ctx->staging);
  const int cur = ctx->cur;
  float* qi = ctx->q[cur];
  float* qo = ctx->q[1 - cur];
  StepArgs a{};
  a.E = ctx->EV;
  a.F = ctx->F;
  a.has_boundary = ctx->F > ctx->F_interior;
  a.q_in = qi;
  a.q_out = qo;
  a.d = ctx->d;
  a.cp = ctx->cp;
  a.ff = ctx->ff;
  a.faces = ctx->faces;
  a.elem_face = ctx->elem_face;
  a.grid_pred = ctx->grid_pred;
  a.grid_face = ctx->grid_face;
  a.grid_corr = ctx->grid_corr;
  a.law = ctx->law;
  a.picard_iters = ctx->picard_iters;
  a.wait_limit = ctx->wait_limit;
  a.wait_limit_set = ctx->wait_limit >= 0;
  a.geom = ctx->geom;
  a.mat = ctx->matf;
  a.nbr = ctx->nbr;
  a.tables = ctx->tables;
  a.dt = static_cast<float>(dt);
  a.status = ctx->status;
  auto part = [&](int k) {
    const int64_t e0 = cb[static_cast<size_t>(k)];
    StepArgs c = a;
    c.E = cb[static_cast<size_t>(k) + 1] - e0;
    c.q_in = qi + e0 * qs;
    c.q_out = qo + e0 * qs;
    c.d = a.d + e0 * ds;
    c.cp = a.cp + e0;
    c.geom = a.geom + e0;
    c.mat = a.mat + e0;
    c.nbr = a.nbr + e0 * 4;
    c.elem_face = a.elem_face + e0 * 4;
    return c;
  };
  DG_CUDA(ctx, cudaMemsetAsync(ctx->status, 0, sizeof(unsigned), ctx->stream));
  // the copies may not touch the staging buffer before earlier work on it is done
  DG_CUDA(ctx, cudaEventRecord(evStart, ctx->stream));
  DG_CUDA(ctx, cudaStreamWaitEvent(ctx->copy_stream, evStart, 0));
  for (int k = 0; k < C; ++k) {
    const int64_t e0 = cb[static_cast<size_t>(k)], ne = cb[static_cast<size_t>(k) + 1] - e0;
    DG_CUDA(ctx, cudaMemcpyAsync(staging + e0 * row, q_in + e0 * row, sizeof(float) * row * ne,
                                 cudaMemcpyHostToDevice, ctx->copy_stream));
    DG_CUDA(ctx, cudaEventRecord(evH[k], ctx->copy_stream));
  }
  // a range of the flux list (element indices in its records stay global); every range runs
  // the kernel of the whole list, so that the fluxes are bitwise those of dg_step
  auto faces_part = [&](int64_t f0, int64_t f1) {
    StepArgs c = a;
    c.faces = a.faces + f0;
    c.ff = a.ff + f0 * ff_stride(ctx->N);
    c.F = f1 - f0;
    return c;
  };
  int64_t launches = 0;
  int faces_done = 0;                       // chunks whose interior faces are launched
  for (int k = 0; k < C; ++k) {
    const StepArgs c = part(k);
    const int64_t e0 = cb[static_cast<size_t>(k)];
    DG_CUDA(ctx, cudaStreamWaitEvent(ctx->stream, evH[k], 0));
    DG_CUDA(ctx, launch_state_in(ctx->N, c.E, 1, staging + e0 * row, 0, qi + e0 * qs, ctx->stream));
    DG_CUDA(ctx, launch_predictor(ctx->N, c, ctx->stream));
    launches += 1;
    if (c.picard_iters > 0) {
      DG_CUDA(ctx, launch_picard(ctx->N, c, ctx->stream));
      ++launches;
    }
    if (!face_ranges) continue;
    // the faces whose both sides are predicted run while later chunks are still uploading
    const HostChunkFaces& hk = ctx->host_faces[static_cast<size_t>(k)];
    if (hk.fb1 > hk.fb0) {
      DG_CUDA(ctx, launch_faces(ctx->N, faces_part(hk.fb0, hk.fb1), ctx->stream));
      ++launches;
    }
    for (; faces_done < C && ctx->host_faces[static_cast<size_t>(faces_done)].need <= k; ++faces_done) {
      const HostChunkFaces& hj = ctx->host_faces[static_cast<size_t>(faces_done)];
      if (hj.fi1 > hj.fi0) {
        DG_CUDA(ctx, launch_faces(ctx->N, faces_part(hj.fi0, hj.fi1), ctx->stream));
        ++launches;
      }
    }
  }
  if (!face_ranges) {
    DG_CUDA(ctx, launch_faces(ctx->N, a, ctx->stream));
    ++launches;
  }
  for (int k = 0; k < C; ++k) {
    const StepArgs c = part(k);
    const int64_t e0 = cb[static_cast<size_t>(k)];
    DG_CUDA(ctx, launch_corrector(ctx->N, c, ctx->stream));
    ++launches;
    if (nsrc > 0) {
      DG_CUDA(ctx, launch_sources_range(ctx->N, nsrc, ctx->source_dev, ctx->amp_dev, 0, qo, e0, e0 + c.E, ctx->stream));
      ++launches;
    }
    DG_CUDA(ctx, launch_state_out(ctx->N, c.E, 1, qo + e0 * qs, staging + e0 * row, 0, ctx->stream));
    DG_CUDA(ctx, cudaEventRecord(evC[k], ctx->stream));
  }
  for (int k = 0; k < C; ++k) {
    const int64_t e0 = cb[static_cast<size_t>(k)], ne = cb[static_cast<size_t>(k) + 1] - e0;
    DG_CUDA(ctx, cudaStreamWaitEvent(ctx->copy_stream, evC[k], 0));
    DG_CUDA(ctx, cudaMemcpyAsync(q_out + e0 * row, staging + e0 * row, sizeof(float) * row * ne,
                                 cudaMemcpyDeviceToHost, ctx->copy_stream));
  }
  if (R > 0 && ctx->n_rec < 65536) {
    DG_CUDA(ctx, launch_receivers(ctx->N, R, ctx->rec_dev, qo, ctx->traces + 3 * R * ctx->n_rec, ctx->stream));
    ++ctx->n_rec;
    ++launches;
  }
  DG_CUDA(ctx, cudaMemcpyAsync(ctx->status_host, ctx->status, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->stream));
  DG_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  DG_CUDA(ctx, cudaStreamSynchronize(ctx->copy_stream));
  ctx->cur = 1 - cur;
  ctx->has_state = true;
  ctx->t += dt;
  ctx->stats.steps += 1;
  ctx->stats.kernel_launches += launches;
  ctx->stats.element_updates += ctx->EV;
  const unsigned st = *ctx->status_host;
  if (st & kStatusNonFinite) return fail(ctx, DG_E_NONFINITE, "non-finite value in the state");
  if (st & kStatusNonHyperbolic) return fail(ctx, DG_E_NONHYPERBOLIC, "effective moduli lost hyperbolicity");
  if (st & kStatusIndex) return fail(ctx, DG_E_MESH, "neighbour index out of range");
  if (st & kStatusTimeout) return fail(ctx, DG_E_CUDA, "a bounded wait on the tensor cores timed out");
  return DG_OK;
}

// ---------------------------------------------------------------------------
// Discrete adjoint with binomial checkpointing
// ---------------------------------------------------------------------------
dg_status dg_adjoint_gradient(dg_ctx* ctx, int64_t n_steps, double dt, const float* ref, int snapshots,
                              double* misfit, double* grad_xi0, double* grad_cd, double* grad_q0,
                              dg_adjoint_info* info) {
  if (!ctx) return fail(ctx, DG_E_ARG, "NULL context");
  if (n_steps < 1 || n_steps > (int64_t(1) << 20)) return fail(ctx, DG_E_ARG, "n_steps must be in 1..2^20");
  if (!ref || !misfit) return fail(ctx, DG_E_ARG, "NULL reference traces or misfit");
  if (snapshots < 0 || snapshots > 4096) return fail(ctx, DG_E_ARG, "snapshots must be in 0..4096");
  if (!ctx->has_material || !ctx->has_state) return fail(ctx, DG_E_STATE, "material and state must be set");
  if (ctx->law != 0) return fail(ctx, DG_E_UNSUPPORTED, "the adjoint covers the CDM law");
  if (ctx->picard_iters > 0) return fail(ctx, DG_E_UNSUPPORTED, "the adjoint covers the CK predictor");
  if (ctx->M != 1) return fail(ctx, DG_E_UNSUPPORTED, "the adjoint covers one member");
  const int R = static_cast<int>(ctx->rec_host.size());
  if (R < 1) return fail(ctx, DG_E_STATE, "the misfit needs receivers (dg_receivers)");
  if (dt <= 0) dt = ctx->dt_cfl;
  if (!std::isfinite(dt)) return fail(ctx, DG_E_ARG, "non-finite dt");
  if (snapshots == 0) {
    // as many state copies as 80 % of the free device memory holds beside the call's other
    // buffers, at most the whole history
    size_t free_b = 0, total_b = 0;
    DG_CUDA(ctx, cudaMemGetInfo(&free_b, &total_b));
    const double state_b = 4.0 * static_cast<double>(ctx->EV) * q_stride(ctx->N);
    const double fit = (0.8 * static_cast<double>(free_b) - 6.0 * state_b -
                        8.0 * static_cast<double>(ctx->F) * adj_rec_stride(ctx->N)) / state_b;
    snapshots = static_cast<int>(std::max(1.0, std::min({fit, static_cast<double>(n_steps + 1), 4096.0})));
  }
  snapshots = static_cast<int>(std::min<int64_t>(snapshots, n_steps + 1));   // more slots are never used
  const int s_free = snapshots - 1;
  if (revolve_cost(n_steps, s_free) > kMaxRevolveSteps)
    return fail(ctx, DG_E_ARG, "too few snapshots for this many steps");
  int64_t fw_plan = 0;
  const std::vector<RevolveAction> plan = revolve_plan(n_steps, snapshots, &fw_plan);
  {
    dg_status st = prepare_steps(ctx, n_steps, dt);
    if (st != DG_OK) return st;
  }
  const int N = ctx->N;
  const int64_t E = ctx->EV, QS = q_stride(N);
  const size_t state_bytes = sizeof(float) * static_cast<size_t>(E * QS);
  const int nsrc = static_cast<int>(ctx->source_host.size());

  // device buffers of the call: snapshot slots, two current states, the state after the
  // last step, two adjoint states, face records, gradients, misfit, reference traces
  std::vector<void*> bufs;
  auto take = [&](size_t bytes) -> void* {
    void* p = dev_alloc(ctx, bytes);
    if (p) bufs.push_back(p);
    return p;
  };
  auto release = [&]() {
    for (void* p : bufs) dev_free(ctx, p);
    bufs.clear();
  };
  float* slots = static_cast<float*>(take(state_bytes * static_cast<size_t>(snapshots)));
  float* work[2] = {static_cast<float*>(take(state_bytes)), static_cast<float*>(take(state_bytes))};
  float* last = static_cast<float*>(take(state_bytes));
  float* lam[2] = {static_cast<float*>(take(state_bytes)), static_cast<float*>(take(state_bytes))};
  float* rec = static_cast<float*>(take(sizeof(float) * static_cast<size_t>(ctx->F * 2 * adj_rec_stride(N))));
  double* g = static_cast<double*>(take(sizeof(double) * static_cast<size_t>(2 * E + 1)));
  float* ref_dev = static_cast<float*>(take(sizeof(float) * static_cast<size_t>(n_steps * R * 3)));
  if (!slots || !work[0] || !work[1] || !last || !lam[0] || !lam[1] || !rec || !g || !ref_dev) {
    release();
    return fail(ctx, DG_E_OOM, "adjoint buffers");
  }
  double* g_xi0 = g;
  double* g_cd = g + E;
  double* J = g + 2 * E;
#define ADJ_CUDA(call)                                         \
  do {                                                         \
    cudaError_t e_ = (call);                                   \
    if (e_ != cudaSuccess) {                                   \
      release();                                               \
      return cuda_fail(ctx, e_, #call);                        \
    }                                                          \
  } while (0)
  ADJ_CUDA(cudaMemcpyAsync(ref_dev, ref, sizeof(float) * n_steps * R * 3, cudaMemcpyHostToDevice, ctx->stream));
  ADJ_CUDA(cudaMemsetAsync(g, 0, sizeof(double) * (2 * E + 1), ctx->stream));
  ADJ_CUDA(cudaMemsetAsync(lam[0], 0, state_bytes, ctx->stream));
  ADJ_CUDA(cudaMemsetAsync(ctx->status, 0, sizeof(unsigned), ctx->stream));
  ADJ_CUDA(cudaMemcpyAsync(slots, ctx->q[ctx->cur], state_bytes, cudaMemcpyDeviceToDevice, ctx->stream));

  StepArgs a{};
  a.E = E;
  a.F = ctx->F;
  a.has_boundary = ctx->F > ctx->F_interior;
  a.d = ctx->d;
  a.cp = ctx->cp;
  a.ff = ctx->ff;
  a.faces = ctx->faces;
  a.elem_face = ctx->elem_face;
  a.grid_pred = ctx->grid_pred;
  a.grid_face = ctx->grid_face;
  a.grid_corr = ctx->grid_corr;
  a.law = 0;
  a.picard_iters = 0;
  a.wait_limit = ctx->wait_limit;
  a.wait_limit_set = ctx->wait_limit >= 0;
  a.geom = ctx->geom;
  a.mat = ctx->matf;
  a.nbr = ctx->nbr;
  a.tables = ctx->tables;
  a.dt = static_cast<float>(dt);
  a.status = ctx->status;
  AdjArgs b{};
  b.E = E;
  b.F = ctx->F;                       // interior faces, then boundary faces
  b.d = ctx->d;
  b.cp = ctx->cp;
  b.rec = rec;
  b.g_xi0 = g_xi0;
  b.g_cd = g_cd;
  b.geom = ctx->geom;
  b.mat = ctx->matf;
  b.faces = ctx->faces;
  b.elem_face = ctx->elem_face;
  b.tables = ctx->tables;
  b.dt = static_cast<float>(dt);

  int64_t launches = 0;
  // one forward step of the state in `in` (step index s) into `out`
  auto forward = [&](const float* in, float* out, int64_t s) -> cudaError_t {
    a.q_in = in;
    a.q_out = out;
    cudaError_t e = launch_predictor(N, a, ctx->stream);
    if (e == cudaSuccess) e = launch_faces(N, a, ctx->stream);
    if (e == cudaSuccess) e = launch_corrector(N, a, ctx->stream);
    launches += 3;
    if (e == cudaSuccess && nsrc > 0) {
      e = launch_sources(N, nsrc, ctx->source_dev, ctx->amp_dev, s, out, ctx->stream);
      ++launches;
    }
    return e;
  };
  // per-action timing (info requested): one event after each action
  struct Events {                        // destroyed on every return path
    std::vector<cudaEvent_t> v;
    ~Events() {
      for (cudaEvent_t e : v)
        if (e) cudaEventDestroy(e);
    }
  } ev_list;
  std::vector<cudaEvent_t>& evs = ev_list.v;
  if (info) {
    evs.assign(plan.size() + 1, nullptr);
    for (auto& ev : evs) ADJ_CUDA(cudaEventCreate(&ev));
    ADJ_CUDA(cudaEventRecord(evs[0], ctx->stream));
  }
  int cb = 0;
  int64_t cur_step = -1, fw_done = 0, adj_done = 0;
  int li = 0;                       // lam[li] holds dJ/dQ^{j+1} before the adjoint of step j
  bool seeded = false;
  for (size_t ai = 0; ai < plan.size(); ++ai) {
    const RevolveAction& act = plan[ai];
    switch (act.kind) {
      case kRestore:
        if (cur_step != act.b) {
          ADJ_CUDA(cudaMemcpyAsync(work[cb], slots + static_cast<size_t>(act.a) * E * QS, state_bytes,
                                   cudaMemcpyDeviceToDevice, ctx->stream));
          cur_step = act.b;
        }
        break;
      case kStore:
        ADJ_CUDA(cudaMemcpyAsync(slots + static_cast<size_t>(act.a) * E * QS, work[cb], state_bytes,
                                 cudaMemcpyDeviceToDevice, ctx->stream));
        break;
      case kAdvance:
        for (int64_t s = act.a; s < act.b; ++s) {
          ADJ_CUDA(forward(work[cb], work[1 - cb], s));
          cb = 1 - cb;
          ++fw_done;
        }
        cur_step = act.b;
        break;
      case kAdjoint: {
        const int64_t j = act.a;
        if (!seeded) {
          // the state after the last step and its misfit term seed dJ/dQ^n
          ADJ_CUDA(forward(work[cb], last, j));
          ++fw_done;
          ADJ_CUDA(launch_misfit(N, R, ctx->rec_dev, last, ref_dev + (n_steps - 1) * R * 3, static_cast<float>(dt),
                                 J, lam[li], ctx->stream));
          ++launches;
          seeded = true;
        }
        a.q_in = work[cb];
        ADJ_CUDA(launch_predictor(N, a, ctx->stream));
        b.q = work[cb];
        b.lam_in = lam[li];
        b.lam_out = lam[1 - li];
        ADJ_CUDA(launch_adjoint(N, b, ctx->stream));
        launches += 3;
        if (j >= 1) {
          ADJ_CUDA(launch_misfit(N, R, ctx->rec_dev, work[cb], ref_dev + (j - 1) * R * 3, static_cast<float>(dt), J,
                                 lam[1 - li], ctx->stream));
          ++launches;
        }
        li = 1 - li;
        ++adj_done;
        break;
      }
    }
    if (info) ADJ_CUDA(cudaEventRecord(evs[ai + 1], ctx->stream));
  }
  // results
  double Jh = 0.0;
  ADJ_CUDA(cudaMemcpyAsync(&Jh, J, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  if (grad_xi0) ADJ_CUDA(cudaMemcpyAsync(grad_xi0, g_xi0, sizeof(double) * E, cudaMemcpyDeviceToHost, ctx->stream));
  if (grad_cd) ADJ_CUDA(cudaMemcpyAsync(grad_cd, g_cd, sizeof(double) * E, cudaMemcpyDeviceToHost, ctx->stream));
  if (grad_q0) {
    const size_t n = static_cast<size_t>(E) * kFields * ctx->L;
    dg_status st = ensure_staging(ctx, n * 8);
    if (st != DG_OK) {
      release();
      return st;
    }
    ADJ_CUDA(launch_state_out(N, ctx->E, 1, lam[li], ctx->staging, 1, ctx->stream));
    ADJ_CUDA(cudaMemcpyAsync(grad_q0, ctx->staging, n * 8, cudaMemcpyDeviceToHost, ctx->stream));
  }
  ADJ_CUDA(cudaMemcpyAsync(ctx->status_host, ctx->status, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->stream));
  ADJ_CUDA(cudaStreamSynchronize(ctx->stream));
  if (info) {
    info->forward_steps = fw_done;
    info->adjoint_steps = adj_done;
    info->forward_ms = info->adjoint_ms = info->copy_ms = 0.0;
    for (size_t ai = 0; ai < plan.size(); ++ai) {
      float ms = 0.f;
      ADJ_CUDA(cudaEventElapsedTime(&ms, evs[ai], evs[ai + 1]));
      const int k = plan[ai].kind;
      if (k == kAdvance) info->forward_ms += ms;
      else if (k == kAdjoint) info->adjoint_ms += ms;
      else info->copy_ms += ms;
    }
  }
#undef ADJ_CUDA
  release();
  *misfit = Jh;
  ctx->stats.kernel_launches += launches;
  const unsigned st = *ctx->status_host;
  if (st & kStatusNonFinite) return fail(ctx, DG_E_NONFINITE, "non-finite value in the state");
  if (st & kStatusNonHyperbolic) return fail(ctx, DG_E_NONHYPERBOLIC, "effective moduli lost hyperbolicity");
  if (st & kStatusIndex) return fail(ctx, DG_E_MESH, "neighbour index out of range");
  if (st & kStatusTimeout) return fail(ctx, DG_E_CUDA, "a bounded wait on the tensor cores timed out");
  return DG_OK;
}

}  // extern "C"

namespace dg {

// Accessors used by the allocation-free step (dg_noalloc.cu).
bool noalloc_view(const dg_ctx* ctx, NoAllocView* v) {
  if (!ctx || !v) return false;
  v->N = ctx->N;
  v->E = ctx->EV;
  v->M = ctx->M;
  v->stream = ctx->stream;
  v->geom = ctx->geom;
  v->mat = ctx->matf;
  v->nbr = ctx->nbr;
  v->faces = ctx->faces;
  v->elem_face = ctx->elem_face;
  v->F = ctx->F;
  v->has_boundary = ctx->F > ctx->F_interior;
  v->tables = ctx->tables;
  v->dt_cfl = ctx->dt_cfl;
  v->has_material = ctx->has_material;
  v->law = ctx->law;
  v->picard_iters = ctx->picard_iters;
  return true;
}

dg_status noalloc_error(dg_ctx* ctx, dg_status s, const char* msg) { return fail(ctx, s, msg); }

cudaError_t launch_predictor(int N, const StepArgs& a, cudaStream_t s) {
  switch (N) {
    case 1: return launch_predictor_t<1>(a, s);
    case 2: return launch_predictor_t<2>(a, s);
    case 3: return launch_predictor_t<3>(a, s);
    case 4: return launch_predictor_t<4>(a, s);
    case 5: return launch_predictor_t<5>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_faces(int N, const StepArgs& a, cudaStream_t s) {
  switch (N) {
    case 1: return launch_faces_t<1>(a, s);
    case 2: return launch_faces_t<2>(a, s);
    case 3: return launch_faces_t<3>(a, s);
    case 4: return launch_faces_t<4>(a, s);
    case 5: return launch_faces_t<5>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_corrector(int N, const StepArgs& a, cudaStream_t s) {
  switch (N) {
    case 1: return launch_corrector_t<1>(a, s);
    case 2: return launch_corrector_t<2>(a, s);
    case 3: return launch_corrector_t<3>(a, s);
    case 4: return launch_corrector_t<4>(a, s);
    case 5: return launch_corrector_t<5>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_picard(int N, const StepArgs& a, cudaStream_t s) {
  switch (N) {
    case 1: return launch_picard_t<1>(a, s);
    case 2: return launch_picard_t<2>(a, s);
    case 3: return launch_picard_t<3>(a, s);
    case 4: return launch_picard_t<4>(a, s);
    case 5: return launch_picard_t<5>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace dg
