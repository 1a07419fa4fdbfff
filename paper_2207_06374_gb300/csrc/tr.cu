// The paper's optimisation procedure on one frame (arXiv 2207.06374, Sec.
// "Optimization procedure"; Algorithm "TRSTMI optimization steps", step 2):
// for each smoothing parameter delta_k in turn, trust-region iterations on
// the smooth maximum F_{s,delta_k} of the variable V, each step from
// CG-Steihaug (Algorithm "Trust-Region CG-Steihaug", after Nocedal and Wright
// Alg. 7.2), the previous stage's result starting the next.
//
// All vectors (the variable, gradient, CG iterates) stay on the device in
// binary64; F and its gradient come from the smooth-maximum kernels (lse.cu),
// Hessian products from a central difference of that exact gradient
// (Hessian-free, as in Nocedal and Wright's Newton-CG), the inner products
// from one-CTA reductions in a fixed order.  The host runs the scalar logic
// (step lengths, the radius rule, accept / reject) on the reduced values it
// reads back, so the whole procedure is the plain sequence of the algorithms:
//   trust-region loop (Nocedal and Wright Alg. 4.1): g = grad F; stop the
//   stage when |g| <= gtol; p from CG-Steihaug with eps = min(1/2, sqrt|g|)|g|;
//   rho = (F(V) - F(V + p)) / (-m(p)); radius / 4 if rho < 1/4, doubled
//   (capped) if rho > 3/4 and |p| reached it; accept if rho > eta, then every
//   column of V is divided by its norm (F is unchanged by that).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "kernels.h"

namespace trstmi {

namespace {

constexpr int kDotThreads = 1024;

// out = a x + b y
__global__ void k_axpby(long long n, double a, const double* x, double b, const double* y,
                        double* out) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) out[i] = a * x[i] + b * y[i];
}

// out[0] = x.y, out[1] = x.z, out[2] = z.z (z may be null), one CTA, each
// thread's strided partial then a fixed tree: the same order every call
__global__ void __launch_bounds__(kDotThreads) k_dots(long long n, const double* x,
                                                      const double* y, const double* z,
                                                      double* out) {
  __shared__ double red[3][kDotThreads];
  double a = 0.0, b = 0.0, c = 0.0;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) {
    a += x[i] * y[i];
    if (z) { b += x[i] * z[i]; c += z[i] * z[i]; }
  }
  red[0][threadIdx.x] = a; red[1][threadIdx.x] = b; red[2][threadIdx.x] = c;
  __syncthreads();
  for (int s = kDotThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      red[0][threadIdx.x] += red[0][threadIdx.x + s];
      red[1][threadIdx.x] += red[1][threadIdx.x + s];
      red[2][threadIdx.x] += red[2][threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) { out[0] = red[0][0]; out[1] = red[1][0]; out[2] = red[2][0]; }
}

// every column of the N x d complex frame divided by its norm
__global__ void k_unit_columns(int N, int d, double2* v, uint32_t* bad) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  double2* col = v + (size_t)j * d;
  double s = 0.0;
  for (int i = 0; i < d; ++i) s += col[i].x * col[i].x + col[i].y * col[i].y;
  if (!(s > 0.0)) { *bad = 1u; return; }
  const double r = sqrt(s);
  for (int i = 0; i < d; ++i) col[i] = make_double2(col[i].x / r, col[i].y / r);
}

struct TrDev {
  int N, d;
  long long n;                   // 2 d N
  int num_sms;
  cudaStream_t s;
  double *x, *xn, *g, *p, *r, *dv, *bd, *tmp, *gp, *gm, *out, *dots;
  uint32_t* bad;
  void* lse_scratch;
  int hv_products;

  unsigned grid() const { return (unsigned)((n + 255) / 256); }

  cudaError_t axpby(double a, const double* x1, double b, const double* y1, double* o) {
    k_axpby<<<grid(), 256, 0, s>>>(n, a, x1, b, y1, o);
    return cudaGetLastError();
  }
  // x.y, and with z also x.z and z.z
  cudaError_t dots3(const double* x1, const double* y1, const double* z1, double* host) {
    k_dots<<<1, kDotThreads, 0, s>>>(n, x1, y1, z1, dots);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(host, dots, 3 * sizeof(double),
                                              cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e;
  }
  double dot(const double* x1, const double* y1, cudaError_t* e) {
    double h[3];
    *e = dots3(x1, y1, nullptr, h);
    return h[0];
  }
  // F (and s) at v, gradient into grad (nullable)
  cudaError_t objective(const double* v, double delta, double* grad, double* F, double* smax) {
    cudaError_t e = launch_lse(N, d, 1, v, delta, true, lse_scratch, out, grad, num_sms, s);
    double h[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, out, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    *F = h[0];
    if (smax) *smax = h[1];
    return e;
  }
  // o = B u: |u| (grad F(x + h u/|u|) - grad F(x - h u/|u|)) / (2h)
  cudaError_t hv(const double* u, double delta, double h, double* o) {
    cudaError_t e;
    const double nu = std::sqrt(dot(u, u, &e));
    if (e != cudaSuccess) return e;
    if (!(nu > 0.0)) return cudaMemsetAsync(o, 0, n * sizeof(double), s);
    const double step = h / nu;
    double F;
    if ((e = axpby(1.0, x, step, u, tmp)) != cudaSuccess) return e;
    if ((e = objective(tmp, delta, gp, &F, nullptr)) != cudaSuccess) return e;
    if ((e = axpby(1.0, x, -step, u, tmp)) != cudaSuccess) return e;
    if ((e = objective(tmp, delta, gm, &F, nullptr)) != cudaSuccess) return e;
    ++hv_products;
    return axpby(nu / (2.0 * h), gp, -nu / (2.0 * h), gm, o);
  }
};

// tau >= 0 (pos) or <= 0 with |z + tau d| = radius, from z.z, z.d, d.d
double to_boundary(double zz, double zd, double dd, double radius, bool pos) {
  double disc = zd * zd - dd * (zz - radius * radius);
  if (disc < 0.0) disc = 0.0;
  return pos ? (-zd + std::sqrt(disc)) / dd : (-zd - std::sqrt(disc)) / dd;
}

// CG-Steihaug on m(p) = g.p + p.Bp / 2 over |p| <= radius, as in the
// paper's Algorithm; p in T.p, the model value in *m.
cudaError_t cg_steihaug(TrDev& T, double delta, double h, double radius, double eps, int maxit,
                        double* m_out, int* iters, int* status) {
  cudaError_t e;
  const size_t bytes = T.n * sizeof(double);
  if ((e = cudaMemsetAsync(T.p, 0, bytes, T.s)) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(T.r, T.g, bytes, cudaMemcpyDeviceToDevice, T.s)) != cudaSuccess) return e;
  if ((e = T.axpby(-1.0, T.g, 0.0, T.g, T.dv)) != cudaSuccess) return e;
  double m = 0.0, rr = T.dot(T.r, T.r, &e);
  if (e != cudaSuccess) return e;
  int st = 3, it = 0;
  if (std::sqrt(rr) < eps) {
    st = 0;
  } else {
    for (it = 0; it < maxit; ++it) {
      if ((e = T.hv(T.dv, delta, h, T.bd)) != cudaSuccess) return e;
      double q[3];
      if ((e = T.dots3(T.dv, T.bd, T.r, q)) != cudaSuccess) return e;   // d.Bd, d.r
      const double dbd = q[0], rd = q[1];
      double zq[3];
      if ((e = T.dots3(T.p, T.p, T.dv, zq)) != cudaSuccess) return e;   // z.z, z.d, d.d
      const double zz = zq[0], zd = zq[1], dd = zq[2];
      if (dbd <= 0.0) {
        const double t1 = to_boundary(zz, zd, dd, radius, true);
        const double t2 = to_boundary(zz, zd, dd, radius, false);
        const double m1 = m + t1 * rd + 0.5 * t1 * t1 * dbd;
        const double m2 = m + t2 * rd + 0.5 * t2 * t2 * dbd;
        const double t = m1 <= m2 ? t1 : t2;
        if ((e = T.axpby(1.0, T.p, t, T.dv, T.p)) != cudaSuccess) return e;
        m = m1 <= m2 ? m1 : m2;
        st = 2; ++it;
        break;
      }
      const double alpha = rr / dbd;
      // |z + alpha d|^2 = z.z + 2 alpha z.d + alpha^2 d.d
      const double zn2 = zz + 2.0 * alpha * zd + alpha * alpha * dd;
      if (std::sqrt(std::max(zn2, 0.0)) >= radius) {
        const double t = to_boundary(zz, zd, dd, radius, true);
        if ((e = T.axpby(1.0, T.p, t, T.dv, T.p)) != cudaSuccess) return e;
        m += t * rd + 0.5 * t * t * dbd;
        st = 1; ++it;
        break;
      }
      if ((e = T.axpby(1.0, T.p, alpha, T.dv, T.p)) != cudaSuccess) return e;
      if ((e = T.axpby(1.0, T.r, alpha, T.bd, T.r)) != cudaSuccess) return e;
      m += alpha * rd + 0.5 * alpha * alpha * dbd;
      const double rr_new = T.dot(T.r, T.r, &e);
      if (e != cudaSuccess) return e;
      if (std::sqrt(rr_new) < eps) { st = 0; ++it; break; }
      const double beta = rr_new / rr;
      if ((e = T.axpby(-1.0, T.r, beta, T.dv, T.dv)) != cudaSuccess) return e;
      rr = rr_new;
    }
  }
  *m_out = m;
  *iters = it;
  *status = st;
  return cudaSuccess;
}

}  // namespace

size_t tr_device_bytes(int N, int d) {
  const size_t vec = ((size_t)2 * d * N * sizeof(double) + 255) & ~(size_t)255;
  return 10 * vec + 512 + lse_scratch_bytes(N, d, 1, true);
}

int tr_solve_device(int N, int d, double* v_dev, const trstmi_tr_options& o, void* scratch,
                    int num_sms, cudaStream_t s, trstmi_tr_row* trace, int cap, int* n_rows,
                    int* hv_products) {
  TrDev T;
  T.N = N; T.d = d; T.n = 2LL * d * N; T.num_sms = num_sms; T.s = s; T.hv_products = 0;
  const size_t vec = ((size_t)T.n * sizeof(double) + 255) & ~(size_t)255;
  unsigned char* b = static_cast<unsigned char*>(scratch);
  double** vecs[] = {&T.xn, &T.g, &T.p, &T.r, &T.dv, &T.bd, &T.tmp, &T.gp, &T.gm};
  for (int k = 0; k < 9; ++k) *vecs[k] = reinterpret_cast<double*>(b + k * vec);
  T.out = reinterpret_cast<double*>(b + 9 * vec);
  T.dots = T.out + 4;
  T.bad = reinterpret_cast<uint32_t*>(T.out + 8);
  T.lse_scratch = b + 9 * vec + 512;
  T.x = v_dev;
  const size_t bytes = T.n * sizeof(double);
  int rows = 0;
  cudaError_t e = cudaMemsetAsync(T.bad, 0, sizeof(uint32_t), s);
  auto unit = [&](double* v) -> cudaError_t {
    k_unit_columns<<<(N + 127) / 128, 128, 0, s>>>(N, d, reinterpret_cast<double2*>(v), T.bad);
    cudaError_t e2 = cudaGetLastError();
    uint32_t bad = 0;
    if (e2 == cudaSuccess) e2 = cudaMemcpyAsync(&bad, T.bad, 4, cudaMemcpyDeviceToHost, s);
    if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(s);
    if (e2 == cudaSuccess && bad) return cudaErrorInvalidValue;
    return e2;
  };
  if (e == cudaSuccess) e = unit(T.x);
  for (int k = 0; k < o.n_delta && e == cudaSuccess; ++k) {
    const double delta = o.delta[k];
    double radius = o.radius0;
    for (int it = 0; it < o.max_outer && e == cudaSuccess; ++it) {
      double F, smax, Fn;
      if ((e = T.objective(T.x, delta, T.g, &F, &smax)) != cudaSuccess) break;
      const double gn = std::sqrt(T.dot(T.g, T.g, &e));
      if (e != cudaSuccess) break;
      if (gn <= o.gtol) break;
      const double eps = std::min(0.5, std::sqrt(gn)) * gn;
      double m;
      int cgit, cgst;
      if ((e = cg_steihaug(T, delta, o.fd_step, radius, eps, o.max_cg, &m, &cgit, &cgst)) !=
          cudaSuccess)
        break;
      const double pn = std::sqrt(T.dot(T.p, T.p, &e));
      if (e != cudaSuccess) break;
      if ((e = T.axpby(1.0, T.x, 1.0, T.p, T.xn)) != cudaSuccess) break;
      if ((e = T.objective(T.xn, delta, nullptr, &Fn, nullptr)) != cudaSuccess) break;
      const double pred = -m;
      const double rho = pred > 0.0 ? (F - Fn) / pred : -1.0;
      const double r_used = radius;
      if (rho < 0.25) radius *= 0.25;
      else if (rho > 0.75 && pn >= (1.0 - 1e-12) * radius)
        radius = std::min(2.0 * radius, o.radius_max);
      const bool acc = rho > o.eta;
      if (acc) {
        if ((e = cudaMemcpyAsync(T.x, T.xn, bytes, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
          break;
        if ((e = unit(T.x)) != cudaSuccess) break;
      }
      if (trace && rows < cap) {
        trstmi_tr_row& r = trace[rows];
        r.stage = k; r.iter = it; r.F = F; r.s = smax; r.gnorm = gn; r.radius = r_used;
        r.rho = rho; r.step_norm = pn; r.pred = pred; r.cg_iters = cgit; r.cg_status = cgst;
        r.accepted = acc ? 1 : 0; r.reserved = 0;
      }
      ++rows;
      if (radius < 1e-14) break;
    }
  }
  if (n_rows) *n_rows = rows;
  if (hv_products) *hv_products = T.hv_products;
  if (e == cudaErrorInvalidValue) return TRSTMI_EINVAL;
  return e == cudaSuccess ? TRSTMI_OK : TRSTMI_ECUDA;
}

}  // namespace trstmi
