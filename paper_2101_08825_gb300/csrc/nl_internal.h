// nl_internal.h -- internal declarations of the GB300 nonlocal-assembly library.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <cstdio>
#include <string>

#include "../../include/nl.h"

namespace nlx {

// ---- errors --------------------------------------------------------------------------
nl_status fail(nl_status st, const char* fmt, ...);
nl_status cuda_fail(cudaError_t e, const char* what);
void clear_error();

#define NL_CUDA(call)                                          \
  do {                                                         \
    cudaError_t _e = (call);                                   \
    if (_e != cudaSuccess) return ::nlx::cuda_fail(_e, #call); \
  } while (0)

#define NL_TRY(call)                  \
  do {                                \
    nl_status _s = (call);            \
    if (_s != NL_OK) return _s;       \
  } while (0)

// Raises a kernel's dynamic shared-memory ceiling to the most the device allows next to the
// kernel's static shared memory.  The attribute is global per kernel, so it is only ever set
// to that one value: launches of the same kernel with different sizes from several threads
// cannot race on it.
template <typename F>
nl_status allow_smem(F* kernel, size_t needed) {
  int dev = 0, mx = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&mx, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
    cudaGetLastError();
    return fail(NL_ECUDA, "cannot query the shared-memory limit");
  }
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_fail(e, "cudaFuncGetAttributes");
  }
  const size_t dyn_max = (size_t)mx > fa.sharedSizeBytes ? (size_t)mx - fa.sharedSizeBytes : 0;
  if (needed > dyn_max)
    return fail(NL_EINTERNAL, "a kernel needs %zu bytes of dynamic shared memory (device limit %zu)",
                needed, dyn_max);
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_max);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_fail(e, "cudaFuncSetAttribute");
  }
  return NL_OK;
}

// ---- kernel launch counter (every launch site wraps its grid size in NL_CNT) ----------
void count_launch();
long long launch_count();
#define NL_CNT(grid) (::nlx::count_launch(), (grid))

// Upper bound on the assembly's block buffer for the calling thread (0 = default: 8 GiB or
// a quarter of the free memory).  The serving workers lower it so that concurrent requests
// stay inside the server's memory budget.
extern thread_local size_t g_block_budget;

// ---- device memory ---------------------------------------------------------------------
void* dev_alloc(size_t bytes, cudaStream_t s);
void dev_free(void* p, size_t bytes, cudaStream_t s);

template <typename T>
struct DevBuf {
  T* p = nullptr;
  size_t n = 0;
  cudaStream_t s = nullptr;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { release(); }
  nl_status alloc(size_t count, cudaStream_t stream) {
    release();
    s = stream;
    n = count;
    if (count == 0) return NL_OK;
    p = static_cast<T*>(dev_alloc(count * sizeof(T), stream));
    if (!p) {
      n = 0;
      return fail(NL_ENOMEM, "device allocation of %zu bytes failed", count * sizeof(T));
    }
    return NL_OK;
  }
  void release() {
    if (p) dev_free(p, n * sizeof(T), s);
    p = nullptr;
    n = 0;
  }
  T* release_ownership() {
    T* q = p;
    p = nullptr;
    n = 0;
    return q;
  }
};

// ---- quadrature rules and kernel constants (host) --------------------------------------
struct Rule {
  int n = 0;
  double bary[16][4] = {};
  double w[16] = {};
};
const Rule& rule(int dim);  // degree-5 simplex rule; weights sum to 1
// 3-point Gauss-Legendre on [0, 1] (the 3x3 product rule of the quadrilaterals)
struct GL3 {
  double g[3], w[3];
};
const GL3& gl3();
// Q1 / Q2 basis on the unit square at (s, t), in the node order of nl_mesh_create_quad: the
// vertices (0,0), (1,0), (1,1), (0,1), then (Q2) the edge midpoints (0,1), (1,2), (2,3),
// (3,0) and the centre; products of the 1D Lagrange bases on {0, 1} or {0, 1/2, 1}.
// order 3: the 8-node serendipity element (the Q2 nodes without the centre), on
// (xi, eta) = (2s - 1, 2t - 1) with nodes (xi_a, eta_a): corners
// (1 + xi xi_a)(1 + eta eta_a)(xi xi_a + eta eta_a - 1)/4, edge nodes
// (1 - xi^2)(1 + eta eta_a)/2 or (1 + xi xi_a)(1 - eta^2)/2.
template <typename T>
__host__ __device__ inline void quad_basis(int order, T s, T t, T* phi) {
  if (order == 3) {
    const T x = (T)2 * s - (T)1, y = (T)2 * t - (T)1;
    const T xm = (T)1 - x, xp = (T)1 + x, ym = (T)1 - y, yp = (T)1 + y;
    phi[0] = (T)0.25 * xm * ym * (-x - y - (T)1);
    phi[1] = (T)0.25 * xp * ym * (x - y - (T)1);
    phi[2] = (T)0.25 * xp * yp * (x + y - (T)1);
    phi[3] = (T)0.25 * xm * yp * (-x + y - (T)1);
    phi[4] = (T)0.5 * ((T)1 - x * x) * ym;
    phi[5] = (T)0.5 * xp * ((T)1 - y * y);
    phi[6] = (T)0.5 * ((T)1 - x * x) * yp;
    phi[7] = (T)0.5 * xm * ((T)1 - y * y);
    return;
  }
  if (order == 2) {
    const T ls[3] = {(T)2 * (s - (T)0.5) * (s - (T)1), (T)4 * s * ((T)1 - s), (T)2 * s * (s - (T)0.5)};
    const T lt[3] = {(T)2 * (t - (T)0.5) * (t - (T)1), (T)4 * t * ((T)1 - t), (T)2 * t * (t - (T)0.5)};
    phi[0] = ls[0] * lt[0];
    phi[1] = ls[2] * lt[0];
    phi[2] = ls[2] * lt[2];
    phi[3] = ls[0] * lt[2];
    phi[4] = ls[1] * lt[0];
    phi[5] = ls[2] * lt[1];
    phi[6] = ls[1] * lt[2];
    phi[7] = ls[0] * lt[1];
    phi[8] = ls[1] * lt[1];
  } else {
    phi[0] = ((T)1 - s) * ((T)1 - t);
    phi[1] = s * ((T)1 - t);
    phi[2] = s * t;
    phi[3] = ((T)1 - s) * t;
  }
}

// Node a of a hexahedron as a point (i, j, k) of the lattice {0, 1, 2}^3 of half steps on the
// unit cube, coded i + 3 j + 9 k: the eight vertices (0,0,0), (1,0,0), (1,1,0), (0,1,0),
// (0,0,1), (1,0,1), (1,1,1), (0,1,1) (in half steps, doubled), then the 27-node element's
// twelve edge midpoints, six face centres and the centre, each group in increasing code.
__host__ __device__ constexpr int hex27_code(int a) {
  switch (a) {
    case 0: return 0;   case 1: return 2;   case 2: return 8;   case 3: return 6;
    case 4: return 18;  case 5: return 20;  case 6: return 26;  case 7: return 24;
    case 8: return 1;   case 9: return 3;   case 10: return 5;  case 11: return 7;
    case 12: return 9;  case 13: return 11; case 14: return 15; case 15: return 17;
    case 16: return 19; case 17: return 21; case 18: return 23; case 19: return 25;
    case 20: return 4;  case 21: return 10; case 22: return 12; case 23: return 14;
    case 24: return 16; case 25: return 22; default: return 13;
  }
}

// w times the basis of a hexahedron at (s, t, u) of the unit cube: NB = 8 the trilinear
// functions of the vertices, NB = 27 (Q2) the products L_i(s) L_j(t) L_k(u) of the quadratic
// Lagrange functions on {0, 1/2, 1} for the node at lattice point (i, j, k), NB = 20 the
// serendipity element on (x, y, z) = (2s-1, 2t-1, 2u-1) with node a at (x_a, y_a, z_a) =
// (i-1, j-1, k-1): a vertex (1/8)(1 + x x_a)(1 + y y_a)(1 + z z_a)(x x_a + y y_a + z z_a - 2),
// an edge node with x_a = 0 (1/4)(1 - x^2)(1 + y y_a)(1 + z z_a), likewise along y and z.
template <int NB, typename T>
__host__ __device__ inline void hex_basis(T s, T t, T u, T w, T* phi) {
  if (NB == 20) {
    const T x = (T)2 * s - (T)1, y = (T)2 * t - (T)1, z = (T)2 * u - (T)1;
#pragma unroll
    for (int a = 0; a < 20; a++) {
      const int c = hex27_code(a);
      const int xa = c % 3 - 1, ya = (c / 3) % 3 - 1, za = c / 9 - 1;
      const T fx = xa == 0 ? (T)1 - x * x : (T)1 + (T)xa * x;
      const T fy = ya == 0 ? (T)1 - y * y : (T)1 + (T)ya * y;
      const T fz = za == 0 ? (T)1 - z * z : (T)1 + (T)za * z;
      if (a < 8)
        phi[a] = (T)0.125 * w * fx * fy * fz * ((T)xa * x + (T)ya * y + (T)za * z - (T)2);
      else
        phi[a] = (T)0.25 * w * fx * fy * fz;
    }
    return;
  }
  if (NB == 8) {
#pragma unroll
    for (int a = 0; a < 8; a++) {
      const int c = hex27_code(a);
      phi[a] = w * ((c % 3) ? s : (T)1 - s) * (((c / 3) % 3) ? t : (T)1 - t) * ((c / 9) ? u : (T)1 - u);
    }
    return;
  }
  const T h = (T)0.5;
  const T ls[3] = {(T)2 * (s - h) * (s - (T)1), (T)4 * s * ((T)1 - s), (T)2 * s * (s - h)};
  const T lt[3] = {(T)2 * (t - h) * (t - (T)1), (T)4 * t * ((T)1 - t), (T)2 * t * (t - h)};
  const T lu[3] = {(T)2 * w * (u - h) * (u - (T)1), (T)4 * w * u * ((T)1 - u), (T)2 * w * u * (u - h)};
  T st[9];
#pragma unroll
  for (int j = 0; j < 3; j++)
#pragma unroll
    for (int i = 0; i < 3; i++) st[i + 3 * j] = ls[i] * lt[j];
#pragma unroll
  for (int a = 0; a < 27; a++) {
    const int c = hex27_code(a);
    phi[a] = st[c % 9] * lu[c / 9];
  }
}
double kernel_constant(int dim, int kernel, double delta, double eps);

// Uploads the rule tables to the current device once.
nl_status ensure_device_tables();

// ---- kernels shared between translation units -------------------------------------------
// Exclusive scan of n int64 counts into out[0..n] (out[n] = total), on stream s.
nl_status exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s);
nl_status exclusive_scan_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, cudaStream_t s);

}  // namespace nlx

// ---- handles -------------------------------------------------------------------------------
struct nl_mesh {
  std::atomic<int> refs{1};
  int dim = 0;
  int order = 1;                   // 1: P1 / Q1, 2: P2 triangles / Q2 quadrilaterals
  int cell = 0;                    // 0: simplices, 1: quadrilaterals (dim 2), 2: hexahedra (dim 3)
  int nb = 0;                      // nodes per element: dim+1 (P1) or 6 (P2)
  int64_t n_vert = 0, n_elem = 0;  // n_vert counts every node
  cudaStream_t stream = nullptr;
  double* coords = nullptr;        // [dim][n_vert]
  int32_t* conn = nullptr;         // [n_elem][nb]: vertices first, then (P2) edge nodes
  uint8_t* elem_in_omega = nullptr;
  uint8_t* node_free = nullptr;
  double* evert = nullptr;         // [n_elem][dim+1, 4 or 8][dim] vertex coordinates per element
  double* blo = nullptr;           // [n_elem][dim] bounding boxes
  double* bhi = nullptr;
  double* vol = nullptr;           // [n_elem]
  double* jinv = nullptr;          // [n_elem][dim][dim]: lambda_{1..dim} = jinv (x - v0)
  float* ef = nullptr;             // [n_elem][EF_STRIDE(dim)]: FP32 vertex offsets v_a - v_0
                                   // (a = 1..dim), inverse Jacobian, volume, v_0 as hi + lo
  int32_t max_conn_deg = 0;
  int64_t* n2e_off = nullptr;      // [n_vert+1] node -> elements
  int32_t* n2e = nullptr;          // [nb n_elem]
  double bb_lo[3] = {0, 0, 0}, bb_hi[3] = {0, 0, 0};
  double max_ext = 0.0;            // largest bounding-box side of an element
  size_t bytes = 0;
};

struct nl_pairs {
  std::atomic<int> refs{1};
  nl_mesh* mesh = nullptr;
  double delta = 0.0, eps = 0.0;
  int64_t n_pairs = 0, nnz = 0;
  int64_t* pair_off = nullptr;  // [n_elem+1]
  int32_t* pair_l = nullptr;    // [n_pairs]
  int64_t* row_ptr = nullptr;   // [n_vert+1]
  int32_t* col = nullptr;       // [nnz]
  int32_t max_pairs_per_elem = 0;
  int32_t max_row_nnz = 0;
  size_t bytes = 0;
};

struct nl_matrix {
  nl_pairs* pairs = nullptr;  // holds a reference
  double* values = nullptr;   // [nnz]
  cudaStream_t stream = nullptr;
};

struct nl_vector {
  nl_mesh* mesh = nullptr;  // holds a reference
  double* v = nullptr;      // [n_vert]
  int64_t n = 0;
  cudaStream_t stream = nullptr;
};

// FP32 per-element record: dim*dim offsets v_a - v_0 (a = 1..dim), dim*dim inverse Jacobian,
// volume, then v_0 as a float-float pair (dim high parts, dim low parts: v_0 = hi + lo to
// about 2^-48 relative), zero padding to a multiple of 16 bytes
#define NL_EF_STRIDE(dim) ((dim) == 2 ? 16 : 32)
#define NL_EF_V0HI(dim) (2 * (dim) * (dim) + 1)
#define NL_EF_V0LO(dim) (2 * (dim) * (dim) + 1 + (dim))

namespace nlx {
void mesh_release(nl_mesh* m);
void pairs_release(nl_pairs* p);
// Builds the pair lists and the CSR pattern (nl_pairs.cu).
nl_status build_pairs(nl_mesh* m, double delta, double eps, nl_pairs* out);
// Runs the assembly kernels (nl_quad.cu); values must hold nnz doubles.
nl_status assemble_values(nl_mesh* m, nl_pairs* p, const nl_kernel_params* kp,
                          const nl_quad_params* qp, nl_precision prec, double* values,
                          nl_assemble_stats* st);
// The same for meshes of hexahedra (nl_quad_hex.cu).
nl_status assemble_values_hex(nl_mesh* m, nl_pairs* p, const nl_kernel_params* kp,
                              const nl_quad_params* qp, nl_precision prec, double* values,
                              nl_assemble_stats* st);
// The same for meshes of quadrilaterals (nl_quad_quad.cu).
nl_status assemble_values_quad(nl_mesh* m, nl_pairs* p, const nl_kernel_params* kp,
                               const nl_quad_params* qp, nl_precision prec, double* values,
                               nl_assemble_stats* st);
// The same for meshes of P2 tetrahedra (nl_quad_p2t.cu).
nl_status assemble_values_p2t(nl_mesh* m, nl_pairs* p, const nl_kernel_params* kp,
                              const nl_quad_params* qp, nl_precision prec, double* values,
                              nl_assemble_stats* st);
// The same for meshes of P2 triangles (nl_quad_p2.cu).
nl_status assemble_values_p2(nl_mesh* m, nl_pairs* p, const nl_kernel_params* kp,
                             const nl_quad_params* qp, nl_precision prec, double* values,
                             nl_assemble_stats* st);
// The same for NL_PREC_MIXED_TF32 / NL_PREC_MIXED_BF16 (nl_quad_mma.cu).
nl_status assemble_values_mma(nl_mesh* m, nl_pairs* p, const nl_kernel_params* kp,
                              const nl_quad_params* qp, nl_precision prec, double* values,
                              nl_assemble_stats* st);
// Right-hand side, operator application and solver kernels (nl_solve.cu).
nl_status apply_matrix(const nl_matrix* A, const double* x, double* y);
nl_status rhs_values(nl_mesh* m, nl_matrix* A, const double* f_nodes, double f_const,
                     const double* g_nodes, double* F);
nl_status solve_system(nl_matrix* A, const nl_vector* rhs, const double* g_nodes, int solver,
                       double rtol, int max_iter, nl_precision prec, double* u_out, int* iters,
                       double* rel_res);
}  // namespace nlx
