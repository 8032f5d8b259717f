// FP64 oracle for the MemGS splatting + voxel-merge hot path.
//
// TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the CPU
// baseline of the benchmark, never by the CUDA library.  It is written for a
// reader checking it against the paper by eye: every step follows the order of
// Sec. II-C (Eq. 1-2), Sec. II-E (Eq. 11) and Sec. II-D (Eq. 3-10); there is no
// blocking or fusion beyond binning Gaussians into the tiles their extent covers,
// which is the definition of which Gaussians a pixel sees.
#include "oracle.h"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <map>
#include <thread>
#include <tuple>
#include <type_traits>
#include <vector>

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr int kTile = 16;                 // tile edge in pixels
constexpr double kAlphaMin = 1.0 / 255.0; // skip a Gaussian whose alpha is below this
constexpr double kAlphaMax = 0.99;        // alpha is clamped to this
constexpr double kTStop = 1e-4;           // stop a pixel once T falls below this
constexpr double kDilation = 0.3;         // px^2 added to the 2D covariance diagonal
constexpr double kFovClamp = 1.3;         // x/z and y/z clamp factor inside the Jacobian
constexpr double kEps32 = 1.0 / 16777216; // 2^-24, unit roundoff of float32

template <class F>
void parallel_for(int64_t n, int nthreads, F f) {
  if (nthreads <= 0) nthreads = (int)std::max(1u, std::thread::hardware_concurrency());
  if (nthreads == 1 || n < 2) {
    for (int64_t i = 0; i < n; ++i) f(i);
    return;
  }
  std::atomic<int64_t> next(0);
  std::vector<std::thread> pool;
  for (int t = 0; t < nthreads; ++t)
    pool.emplace_back([&] {
      for (;;) {
        int64_t i = next.fetch_add(1);
        if (i >= n) break;
        f(i);
      }
    });
  for (auto& th : pool) th.join();
}

// ---------- small dense linear algebra (row-major) ----------
// Templated on the element types so that the chain rule below also runs on AbsVal.
template <class TA, class TB, class TC>
void matmul(const TA* A, const TB* B, TC* C, int n, int k, int m) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < m; ++j) {
      TC s = TC();
      for (int l = 0; l < k; ++l) s += A[i * k + l] * B[l * m + j];
      C[i * m + j] = s;
    }
}
template <class T>
void transpose(const T* A, T* At, int n, int m) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < m; ++j) At[j * n + i] = A[i * m + j];
}

// Running-error arithmetic for a computation that is linear in its AbsVal inputs: every
// sum and difference adds magnitudes, every product takes |constant|.  Run on the sums
// of |terms| of its inputs, a linear map gives the sum over all its paths of the
// absolute products: the quantity a floating-point evaluation's rounding error is
// proportional to, however much the exact result cancels.
struct AbsVal {
  double v = 0;
};
inline AbsVal operator+(AbsVal a, AbsVal b) { return {a.v + b.v}; }
inline AbsVal operator-(AbsVal a, AbsVal b) { return {a.v + b.v}; }
inline AbsVal operator-(AbsVal a) { return a; }
inline AbsVal operator*(AbsVal a, double c) { return {a.v * std::fabs(c)}; }
inline AbsVal operator*(double c, AbsVal a) { return {a.v * std::fabs(c)}; }
inline AbsVal operator/(AbsVal a, double c) { return {a.v / std::fabs(c)}; }
inline AbsVal& operator+=(AbsVal& a, AbsVal b) { a.v += b.v; return a; }
inline AbsVal& operator*=(AbsVal& a, double c) { a.v *= std::fabs(c); return a; }

// Rotation matrix of a unit quaternion (w, x, y, z).
void quat_to_rot(const double* q, double* R) {
  double w = q[0], x = q[1], y = q[2], z = q[3];
  R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
  R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
  R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

// d(sum_ij G_ij R_ij)/dq for the rotation above, q unit (w, x, y, z).
template <class T>
void rot_backward(const double* q, const T* G, T* dq) {
  double w = q[0], x = q[1], y = q[2], z = q[3];
  dq[0] = 2 * (-z * G[1] + y * G[2] + z * G[3] - x * G[5] - y * G[6] + x * G[7]);
  dq[1] = 2 * (y * G[1] + z * G[2] + y * G[3] - 2 * x * G[4] - w * G[5] + z * G[6] + w * G[7] -
               2 * x * G[8]);
  dq[2] = 2 * (-2 * y * G[0] + x * G[1] + w * G[2] + x * G[3] + z * G[5] - w * G[6] + z * G[7] -
               2 * y * G[8]);
  dq[3] = 2 * (-2 * z * G[0] - w * G[1] + x * G[2] + w * G[3] - 2 * z * G[4] + y * G[5] +
               x * G[6] + y * G[7]);
}

// Cyclic Jacobi eigen-decomposition of a symmetric 3x3: A = V diag(w) V^T.
void eig_sym3(const double* Ain, double* w, double* V) {
  double A[9];
  std::memcpy(A, Ain, sizeof(A));
  for (int i = 0; i < 9; ++i) V[i] = (i % 4 == 0) ? 1.0 : 0.0;
  const int P[3] = {0, 0, 1}, Q[3] = {1, 2, 2};
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = A[1] * A[1] + A[2] * A[2] + A[5] * A[5];
    double dia = A[0] * A[0] + A[4] * A[4] + A[8] * A[8];
    if (off <= 1e-36 * dia || off == 0.0) break;
    for (int r = 0; r < 3; ++r) {
      int p = P[r], q = Q[r];
      double apq = A[p * 3 + q];
      if (apq == 0.0) continue;
      double theta = (A[q * 3 + q] - A[p * 3 + p]) / (2 * apq);
      double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1));
      double c = 1 / std::sqrt(t * t + 1), s = t * c;
      for (int k = 0; k < 3; ++k) {
        double akp = A[k * 3 + p], akq = A[k * 3 + q];
        A[k * 3 + p] = c * akp - s * akq;
        A[k * 3 + q] = s * akp + c * akq;
      }
      for (int k = 0; k < 3; ++k) {
        double apk = A[p * 3 + k], aqk = A[q * 3 + k];
        A[p * 3 + k] = c * apk - s * aqk;
        A[q * 3 + k] = s * apk + c * aqk;
      }
      for (int k = 0; k < 3; ++k) {
        double vkp = V[k * 3 + p], vkq = V[k * 3 + q];
        V[k * 3 + p] = c * vkp - s * vkq;
        V[k * 3 + q] = s * vkp + c * vkq;
      }
    }
  }
  w[0] = A[0]; w[1] = A[4]; w[2] = A[8];
}

// f(A) = V diag(f(w)) V^T for a symmetric positive semi-definite A.
void sym_fun(const double* A, double power, double* out) {
  double w[3], V[9];
  eig_sym3(A, w, V);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0;
      for (int k = 0; k < 3; ++k) s += V[i * 3 + k] * std::pow(std::max(w[k], 0.0), power) * V[j * 3 + k];
      out[i * 3 + j] = s;
    }
}

void inv3(const double* A, double* B) {
  double det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
               A[2] * (A[3] * A[7] - A[4] * A[6]);
  B[0] = (A[4] * A[8] - A[5] * A[7]) / det;
  B[1] = (A[2] * A[7] - A[1] * A[8]) / det;
  B[2] = (A[1] * A[5] - A[2] * A[4]) / det;
  B[3] = (A[5] * A[6] - A[3] * A[8]) / det;
  B[4] = (A[0] * A[8] - A[2] * A[6]) / det;
  B[5] = (A[2] * A[3] - A[0] * A[5]) / det;
  B[6] = (A[3] * A[7] - A[4] * A[6]) / det;
  B[7] = (A[1] * A[6] - A[0] * A[7]) / det;
  B[8] = (A[0] * A[4] - A[1] * A[3]) / det;
}

// ---------- real spherical harmonics from their definition ----------
// Y_lm = K_lm * (d^|m| P_l / dz^|m|)(z) * {Re (x+iy)^m  (m>0), 1 (m=0), Im (x+iy)^|m| (m<0)}
// with K_lm = sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!) and an extra sqrt(2) when m != 0.
struct ShTables {
  double K[16];
  double Q[16][4];  // coefficients of d^|m| P_l / dz^|m| in powers of z
  int l[16], m[16];
  ShTables() {
    double P[4][4] = {};
    P[0][0] = 1;
    P[1][1] = 1;
    for (int L = 1; L < 3; ++L)  // (L+1) P_{L+1} = (2L+1) z P_L - L P_{L-1}
      for (int k = 0; k < 4; ++k) {
        double a = (k > 0 ? (2 * L + 1) * P[L][k - 1] : 0.0) - L * P[L - 1][k];
        P[L + 1][k] = a / (L + 1);
      }
    auto fact = [](int n) { double f = 1; for (int i = 2; i <= n; ++i) f *= i; return f; };
    for (int L = 0; L <= 3; ++L)
      for (int M = -L; M <= L; ++M) {
        int idx = L * L + L + M, am = std::abs(M);
        l[idx] = L; m[idx] = M;
        K[idx] = std::sqrt((2 * L + 1) / (4 * kPi) * fact(L - am) / fact(L + am)) *
                 (M != 0 ? std::sqrt(2.0) : 1.0);
        for (int k = 0; k < 4; ++k) {
          double c = (k + am < 4) ? P[L][k + am] : 0.0;
          for (int d = 0; d < am; ++d) c *= (k + am - d);
          Q[idx][k] = c;
        }
      }
  }
};
const ShTables& sh_tables() {
  static ShTables t;
  return t;
}

void sh_eval(int degree, const double* d, double* Y, double* dY) {
  const ShTables& T = sh_tables();
  int K = (degree + 1) * (degree + 1);
  double x = d[0], y = d[1], z = d[2];
  for (int k = 0; k < K; ++k) {
    int am = std::abs(T.m[k]);
    double q = 0, dq = 0, zp = 1;
    for (int p = 0; p < 4; ++p) {
      q += T.Q[k][p] * zp;
      if (p + 1 < 4) dq += (p + 1) * T.Q[k][p + 1] * zp;
      zp *= z;
    }
    // (x+iy)^am and am*(x+iy)^(am-1)
    double re = 1, im = 0, dre = 0, dim = 0;
    for (int p = 0; p < am; ++p) {
      dre = re; dim = im;  // (x+iy)^(am-1) after the last iteration
      double nre = re * x - im * y, nim = re * y + im * x;
      re = nre; im = nim;
    }
    dre *= am; dim *= am;
    double ang, dang_dx, dang_dy;
    if (T.m[k] > 0) { ang = re; dang_dx = dre; dang_dy = -dim; }
    else if (T.m[k] < 0) { ang = im; dang_dx = dim; dang_dy = dre; }
    else { ang = 1; dang_dx = 0; dang_dy = 0; }
    Y[k] = T.K[k] * q * ang;
    if (dY) {
      dY[k * 3 + 0] = T.K[k] * q * dang_dx;
      dY[k * 3 + 1] = T.K[k] * q * dang_dy;
      dY[k * 3 + 2] = T.K[k] * dq * ang;
    }
  }
}

// ---------- projection (Eq. 1, Eq. 2) ----------
struct Proj {
  bool culled = true;     // near plane or non-positive determinant
  bool visible = false;   // not culled and the rect is non-empty
  double p[3] = {0, 0, 0};
  double qn[4], qnorm, Rq[9], s[3], S3[9];
  double limx, limy, xr, yr;
  bool clampx, clampy;
  double J[6], T[6], cov[3], det, conic[3];
  double u, v, lam, r3;
  double cond = 1;  // conditioning of the exponent's evaluation (see orc_margins)
  int r = 0;
  int rect[4] = {0, 0, -1, -1};
  double o;
  int64_t index = 0;  // of the Gaussian
  double dir[3], vnorm, raw[3], rgb[3];
  // Near-tie alternatives of the tile rect: union and intersection of the rects
  // any near-tie resolution could give (union empty when nothing could be drawn).
  int rect_union[4] = {0, 0, -1, -1};
  int rect_inter[4] = {0, 0, -1, -1};
};

int tiles_x(const orc_camera* c) { return (c->width + kTile - 1) / kTile; }
int tiles_y(const orc_camera* c) { return (c->height + kTile - 1) / kTile; }

void rect_of(double u, double v, int r, const orc_camera* cam, int* rc) {
  int tx = tiles_x(cam), ty = tiles_y(cam);
  rc[0] = std::max(0, (int)std::floor((u - r) / kTile));
  rc[1] = std::max(0, (int)std::floor((v - r) / kTile));
  rc[2] = std::min(tx - 1, (int)std::floor((u + r) / kTile));
  rc[3] = std::min(ty - 1, (int)std::floor((v + r) / kTile));
}
bool rect_empty(const int* rc) { return rc[2] < rc[0] || rc[3] < rc[1]; }
bool in_rect(const int* rc, int x, int y) { return x >= rc[0] && x <= rc[2] && y >= rc[1] && y <= rc[3]; }

void project_one(const orc_gaussians* g, const orc_camera* cam, const orc_margins* mg, int64_t i,
                 Proj& P) {
  const double* mu = g->means + 3 * i;
  const double* Rw = cam->R;
  P.index = i;
  for (int r = 0; r < 3; ++r)
    P.p[r] = Rw[r * 3 + 0] * mu[0] + Rw[r * 3 + 1] * mu[1] + Rw[r * 3 + 2] * mu[2] + cam->t[r];
  double tx = P.p[0], ty = P.p[1], tz = P.p[2];
  bool near_cull = !(tz > cam->near_z);
  bool near_tie = mg && std::fabs(tz - cam->near_z) < mg->near_rel * cam->near_z;
  if (near_cull && !near_tie) return;

  // Eq. 2: Sigma = R S S^T R^T with S = diag(exp(log_scale)), R from the unit quaternion.
  const double* q = g->quats + 4 * i;
  P.qnorm = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  for (int k = 0; k < 4; ++k) P.qn[k] = q[k] / P.qnorm;
  quat_to_rot(P.qn, P.Rq);
  for (int k = 0; k < 3; ++k) P.s[k] = std::exp(g->log_scales[3 * i + k]);
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double acc = 0;
      for (int k = 0; k < 3; ++k) acc += P.Rq[a * 3 + k] * P.s[k] * P.s[k] * P.Rq[b * 3 + k];
      P.S3[a * 3 + b] = acc;
    }
  // Eq. 1: Sigma_I = J W Sigma W^T J^T, J the Jacobian of the perspective map at the mean.
  P.limx = kFovClamp * (0.5 * cam->width / cam->fx);
  P.limy = kFovClamp * (0.5 * cam->height / cam->fy);
  P.xr = tx / tz;
  P.yr = ty / tz;
  P.clampx = P.xr < -P.limx || P.xr > P.limx;
  P.clampy = P.yr < -P.limy || P.yr > P.limy;
  double xc = std::min(P.limx, std::max(-P.limx, P.xr));
  double yc = std::min(P.limy, std::max(-P.limy, P.yr));
  P.J[0] = cam->fx / tz; P.J[1] = 0;               P.J[2] = -cam->fx * xc / tz;
  P.J[3] = 0;            P.J[4] = cam->fy / tz;    P.J[5] = -cam->fy * yc / tz;
  matmul(P.J, Rw, P.T, 2, 3, 3);
  double TS[6], Tt[6], C2[4];
  matmul(P.T, P.S3, TS, 2, 3, 3);
  transpose(P.T, Tt, 2, 3);
  matmul(TS, Tt, C2, 2, 3, 2);
  P.cov[0] = C2[0] + kDilation;
  P.cov[1] = C2[1];
  P.cov[2] = C2[3] + kDilation;
  P.det = P.cov[0] * P.cov[2] - P.cov[1] * P.cov[1];
  if (!(P.det > 0)) return;
  P.conic[0] = P.cov[2] / P.det;
  P.conic[1] = -P.cov[1] / P.det;
  P.conic[2] = P.cov[0] / P.det;
  P.u = cam->fx * tx / tz + cam->cx;
  P.v = cam->fy * ty / tz + cam->cy;
  double mid = 0.5 * (P.cov[0] + P.cov[2]);
  P.lam = mid + std::sqrt(std::max(0.1, mid * mid - P.det));
  {
    double tn = 0, sn = 0;
    for (int k = 0; k < 6; ++k) tn += P.T[k] * P.T[k];
    for (int k = 0; k < 9; ++k) sn += P.S3[k] * P.S3[k];
    double disc = std::sqrt(0.25 * (P.cov[0] - P.cov[2]) * (P.cov[0] - P.cov[2]) + P.cov[1] * P.cov[1]);
    double lmin = mid - disc, kappa = (mid + disc) / lmin;
    double gamma = (tn * std::sqrt(sn) + P.cov[0] + P.cov[2]) / lmin;
    P.cond = std::sqrt(gamma * kappa) + kappa;
  }
  P.r3 = 3.0 * std::sqrt(P.lam);
  P.r = (int)std::ceil(P.r3);
  rect_of(P.u, P.v, P.r, cam, P.rect);
  P.culled = near_cull;
  P.visible = !P.culled && !rect_empty(P.rect);

  // Near-tie alternatives of the extent decision.
  int rs[2] = {P.r, P.r};
  if (mg) {
    double k = std::round(P.r3);
    if (std::fabs(P.r3 - k) < mg->radius_abs) { rs[0] = (int)k; rs[1] = (int)k + 1; }
  }
  int U[4] = {1 << 30, 1 << 30, -(1 << 30), -(1 << 30)};
  int I[4] = {-(1 << 30), -(1 << 30), 1 << 30, 1 << 30};
  const double ctr[2] = {P.u, P.v};
  int lim[2] = {tiles_x(cam) - 1, tiles_y(cam) - 1};
  for (int a = 0; a < 2; ++a) {
    int rr = rs[a];
    for (int ax = 0; ax < 2; ++ax)
      for (int side = 0; side < 2; ++side) {
        double e = side == 0 ? ctr[ax] - rr : ctr[ax] + rr;
        double f = std::floor(e / kTile);
        double lo = f, hi = f;
        if (mg) {
          double b = std::round(e / kTile) * kTile;
          if (std::fabs(e - b) < mg->extent_px) { lo = b / kTile - 1; hi = b / kTile; }
        }
        if (side == 0) {  // lower edge: union takes the smallest, intersection the largest
          U[ax] = std::min(U[ax], std::max(0, (int)lo));
          I[ax] = std::max(I[ax], std::max(0, (int)hi));
        } else {
          U[2 + ax] = std::max(U[2 + ax], std::min(lim[ax], (int)hi));
          I[2 + ax] = std::min(I[2 + ax], std::min(lim[ax], (int)lo));
        }
      }
  }
  std::memcpy(P.rect_union, U, sizeof(U));
  if (near_tie || P.culled) {
    int e[4] = {0, 0, -1, -1};
    std::memcpy(P.rect_inter, e, sizeof(e));
  } else {
    std::memcpy(P.rect_inter, I, sizeof(I));
  }

  P.o = 1.0 / (1.0 + std::exp(-g->opacity_logit[i]));
  // Colour from spherical harmonics in the direction from the camera centre.
  double C[3];
  for (int k = 0; k < 3; ++k)
    C[k] = -(Rw[0 * 3 + k] * cam->t[0] + Rw[1 * 3 + k] * cam->t[1] + Rw[2 * 3 + k] * cam->t[2]);
  double dv[3] = {mu[0] - C[0], mu[1] - C[1], mu[2] - C[2]};
  P.vnorm = std::sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
  for (int k = 0; k < 3; ++k) P.dir[k] = dv[k] / P.vnorm;
  int K = (g->sh_degree + 1) * (g->sh_degree + 1);
  double Y[16];
  sh_eval(g->sh_degree, P.dir, Y, nullptr);
  const double* sh = g->sh + (size_t)i * K * 3;
  for (int ch = 0; ch < 3; ++ch) {
    double acc = 0;
    for (int k = 0; k < K; ++k) acc += sh[k * 3 + ch] * Y[k];
    P.raw[ch] = acc + 0.5;
    P.rgb[ch] = std::max(0.0, P.raw[ch]);
  }
}

std::vector<Proj> project_all(const orc_gaussians* g, const orc_camera* cam, const orc_margins* mg,
                              int nthreads) {
  std::vector<Proj> P(g->n);
  parallel_for((g->n + 1023) / 1024, nthreads, [&](int64_t b) {
    for (int64_t i = b * 1024; i < std::min<int64_t>(g->n, (b + 1) * 1024); ++i) project_one(g, cam, mg, i, P[i]);
  });
  return P;
}

// ---------- binning ----------
struct Entry {
  int32_t g;
  bool included;   // the FP64 decision puts the Gaussian in this tile
  bool uncertain;  // a near-tie could add or remove it
};

std::vector<std::vector<Entry>> bin_tiles(const std::vector<Proj>& P, const orc_camera* cam,
                                          const std::vector<char>& want_tile, int nthreads) {
  int TX = tiles_x(cam), TY = tiles_y(cam);
  std::vector<std::vector<Entry>> bins((size_t)TX * TY);
  for (size_t i = 0; i < P.size(); ++i) {
    const Proj& p = P[i];
    const int* U = p.rect_union;
    if (rect_empty(U)) continue;
    for (int y = U[1]; y <= U[3]; ++y)
      for (int x = U[0]; x <= U[2]; ++x) {
        int t = y * TX + x;
        if (!want_tile[t]) continue;
        bool inc = p.visible && in_rect(p.rect, x, y);
        bool unc = !in_rect(p.rect_inter, x, y);
        if (!inc && !unc) continue;
        bins[t].push_back(Entry{(int32_t)i, inc, unc});
      }
  }
  // Front-to-back order: the float32 rounding of the camera depth, then Gaussian index.
  parallel_for((int64_t)bins.size(), nthreads, [&](int64_t t) {
    std::stable_sort(bins[t].begin(), bins[t].end(), [&](const Entry& a, const Entry& b) {
      float za = (float)P[a.g].p[2], zb = (float)P[b.g].p[2];
      if (za != zb) return za < zb;
      return a.g < b.g;
    });
  });
  return bins;
}

std::vector<char> tile_mask(const orc_camera* cam, const int32_t* tiles, int32_t n_tiles) {
  int n = tiles_x(cam) * tiles_y(cam);
  std::vector<char> want(n, n_tiles < 0 ? 1 : 0);
  for (int i = 0; i < std::max(0, n_tiles); ++i)
    if (tiles[i] >= 0 && tiles[i] < n) want[tiles[i]] = 1;
  return want;
}

// One pixel's front-to-back pass over its tile list (Eq. 11 with the cutoffs).
struct Contribution {
  int32_t g;
  double alpha, a, G, Tb, dx, dy;
  double ma;  // relative alpha margin at this pixel (the modelled float32 error of alpha)
};
struct PixelResult {
  double rgb[3] = {0, 0, 0}, depth = 0, T = 1;
  double t_err = 0;  // modelled relative float32 error of T at the end of the pass
  int n_contrib = 0, n_eval = 0;
  uint8_t flags = 0;
  std::vector<Contribution> contrib;  // only filled when requested
  std::vector<int32_t> touched;       // Gaussians evaluated up to the stop
};

bool near_midpoint(double z, double rel) {
  float f = (float)z;
  double up = 0.5 * ((double)f + (double)std::nextafter(f, 1e30f));
  double dn = 0.5 * ((double)f + (double)std::nextafter(f, -1e30f));
  return std::fabs(z - up) < rel * z || std::fabs(z - dn) < rel * z;
}
bool near_key_tie(double za, double zb, double rel) {
  float fa = (float)za, fb = (float)zb;
  bool close = fb <= std::nextafter(fa, 1e30f) && fa <= std::nextafter(fb, 1e30f);
  return close && (near_midpoint(za, rel) || near_midpoint(zb, rel));
}

double power_at(const Proj& P, double px, double py, double* dx, double* dy) {
  *dx = P.u - px;
  *dy = P.v - py;
  return -0.5 * (P.conic[0] * (*dx) * (*dx) + P.conic[2] * (*dy) * (*dy)) - P.conic[1] * (*dx) * (*dy);
}

// A near-tie decision of one pixel's pass: kind 1 alpha cutoff, 2 T stop, 4 depth order
// (entries k and kp may swap), 8 extent / near plane (entry k may be in or out of the
// tile list).  The opacity clamp (flag 16) is continuous in the image and is not one.
struct Tie {
  uint8_t kind;
  int32_t k, kp;
};

void blend_pixel(const std::vector<Proj>& P, const std::vector<Entry>& list, int px, int py,
                 const orc_margins* mg, bool keep, PixelResult& R, const Tie* flip = nullptr,
                 std::vector<Tie>* ties = nullptr) {
  int pos = 0;  // index among the included entries (the CUDA list position)
  double prev_tz = -1;
  int32_t prev_k = -1;
  double t_var = 0;  // sum of squared relative alpha margins, weighted by alpha/(1-alpha)
  auto flipped = [&](uint8_t kind, size_t k) { return flip && flip->kind == kind && flip->k == (int32_t)k; };
  auto tie = [&](uint8_t kind, size_t k, int32_t kp) {
    if (ties) ties->push_back(Tie{kind, (int32_t)k, kp});
  };
  for (size_t k = 0; k < list.size(); ++k) {
    const Entry& e = list[k];
    const Proj& p = P[e.g];
    double dx, dy, power = power_at(p, px, py, &dx, &dy);
    double a = p.o * std::exp(power);
    double alpha = std::min(kAlphaMax, a);
    double ma = mg ? mg->alpha_rel + mg->cond_rel * p.cond * std::fabs(power) : 0;
    bool potential = power <= 0 && alpha >= kAlphaMin * (1 - ma);
    if (keep && potential) R.touched.push_back(e.g);
    if (mg && e.uncertain && potential) {
      R.flags |= 8;
      tie(8, k, -1);
    }
    if (e.included == flipped(8, k)) continue;
    ++pos;
    if (mg && potential) {
      // The order is decided on float32 depth keys; a pair can swap only when the
      // keys are within one ulp and a depth sits next to a float32 rounding midpoint.
      if (prev_tz >= 0 && near_key_tie(prev_tz, p.p[2], mg->depth_rel)) {
        R.flags |= 4;
        tie(4, k, prev_k);
      }
      prev_tz = p.p[2];
      prev_k = (int32_t)k;
    }
    if (power > 0) continue;
    if (mg && std::fabs(alpha * 255.0 - 1.0) < ma) {
      R.flags |= 1;
      tie(1, k, -1);
    }
    if (mg && std::fabs(a - kAlphaMax) < (mg->clamp_rel + ma) * kAlphaMax) R.flags |= 16;
    if ((alpha < kAlphaMin) != flipped(1, k)) continue;
    double w = alpha * R.T;
    if (keep) R.contrib.push_back(Contribution{e.g, alpha, a, std::exp(power), R.T, dx, dy, ma});
    for (int c = 0; c < 3; ++c) R.rgb[c] += p.rgb[c] * w;
    R.depth += p.p[2] * w;
    R.T = R.T * (1 - alpha);
    R.n_contrib = pos;
    if (mg) {
      double e = alpha / (1 - alpha) * ma;
      t_var += e * e;
      R.t_err = std::sqrt(t_var);
      if (std::fabs(R.T / kTStop - 1) < mg->T_rel + std::sqrt(t_var)) {
        R.flags |= 2;
        tie(2, k, -1);
      }
    }
    if ((R.T < kTStop) != flipped(2, k)) {
      R.n_eval = pos;
      return;
    }
  }
  R.n_eval = pos;
}

// The pixel's image with its one near-tie decision taken the other way.
void blend_pixel_flipped(const std::vector<Proj>& P, const std::vector<Entry>& list, int px, int py,
                         const orc_margins* mg, const Tie& t, PixelResult& R) {
  if (t.kind != 4) {
    blend_pixel(P, list, px, py, mg, false, R, &t, nullptr);
    return;
  }
  std::vector<Entry> swapped(list);  // the two neighbouring contributors in the other order
  std::swap(swapped[t.k], swapped[t.kp]);
  blend_pixel(P, swapped, px, py, mg, false, R, nullptr, nullptr);
}

uint64_t mix(uint64_t h, uint64_t v) {
  h ^= v + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2);
  return h;
}

// Chain rule from the screen-space gradient of one Gaussian to its parameters.
// Parameter gradient of one Gaussian from its screen-space gradient (linear in g2);
// G = double computes it, G = AbsVal its running-error scale.
template <class G>
struct ParamGradT {
  G mu[3] = {}, ls[3] = {}, q[4] = {}, op = G(), sh[48] = {};
  double stat = 0;
  // G = double only: modelled float32 error that comes from the SH direction (see below)
  double xmu[3] = {0, 0, 0}, xsh[48] = {};
};

// The SH argument is the direction from the camera centre to the mean.  A float32
// evaluation forms it from rounded coordinates: model its error as
// dd = 4 x 2^-24 (|mu|_1 + |C|_1) / |mu - C| + 4 x 2^-24 per component, take the change
// of each basis function and of its gradient over dd along each axis (plus 16 x 2^-24
// for evaluating the polynomial), and carry it to the SH and mean gradients.  Where the
// colour clamp max(0, raw) sits within the modelled error of raw, the clamp decision can
// go either way: the whole channel's terms count as error.
void sh_direction_error(const orc_gaussians* g, const orc_camera* cam, const Proj& P, const double* sh, int K,
                        const double* dcol, const double* ddir, const double* Y, const double* dY,
                        ParamGradT<double>& o) {
  double C[3], l1 = 0;
  for (int k = 0; k < 3; ++k) {
    C[k] = -(cam->R[0 * 3 + k] * cam->t[0] + cam->R[1 * 3 + k] * cam->t[1] + cam->R[2 * 3 + k] * cam->t[2]);
    l1 += std::fabs(g->means[3 * P.index + k]) + std::fabs(C[k]);
  }
  const double dd = 4 * kEps32 * l1 / P.vnorm + 4 * kEps32;
  double eY[16] = {}, edY[48] = {};
  for (int a = 0; a < 3; ++a) {
    double d2[3] = {P.dir[0], P.dir[1], P.dir[2]};
    d2[a] += dd;
    double Y2[16], dY2[48];
    sh_eval(g->sh_degree, d2, Y2, dY2);
    for (int k = 0; k < K; ++k) {
      eY[k] += std::fabs(Y2[k] - Y[k]);
      for (int b = 0; b < 3; ++b) edY[k * 3 + b] += std::fabs(dY2[k * 3 + b] - dY[k * 3 + b]);
    }
  }
  for (int k = 0; k < K; ++k) {
    eY[k] += 16 * kEps32;
    for (int b = 0; b < 3; ++b) edY[k * 3 + b] += 16 * kEps32 * (1 + std::fabs(dY[k * 3 + b]));
  }
  double eddir[3] = {0, 0, 0};
  for (int ch = 0; ch < 3; ++ch) {
    double raw_err = 0;
    for (int k = 0; k < K; ++k) raw_err += std::fabs(sh[k * 3 + ch]) * (eY[k] + 16 * kEps32 * std::fabs(Y[k]));
    const bool open = std::fabs(P.raw[ch]) <= raw_err;  // the clamp decision is in doubt
    if (P.raw[ch] < 0 && !open) continue;
    for (int k = 0; k < K; ++k) {
      o.xsh[k * 3 + ch] += std::fabs(dcol[ch]) * (eY[k] + (open ? std::fabs(Y[k]) : 0.0));
      for (int b = 0; b < 3; ++b)
        eddir[b] += std::fabs(dcol[ch] * sh[k * 3 + ch]) * (edY[k * 3 + b] + (open ? std::fabs(dY[k * 3 + b]) : 0.0));
    }
  }
  double e_sum = eddir[0] + eddir[1] + eddir[2];
  double dsum = std::fabs(ddir[0]) + std::fabs(ddir[1]) + std::fabs(ddir[2]);
  for (int a = 0; a < 3; ++a) o.xmu[a] += (eddir[a] + e_sum + 2 * dd * dsum) / P.vnorm;
}

template <class G>
void gaussian_backward_local(const orc_gaussians* g, const orc_camera* cam, const Proj& P, int64_t i,
                             const G* g2, ParamGradT<G>& o) {
  G du = g2[0], dv = g2[1], dA = g2[2], dB = g2[3], dC = g2[4], dop = g2[5];
  const G* dcol = g2 + 6;
  G dd = g2[9];
  double fx = cam->fx, fy = cam->fy;
  double tx = P.p[0], ty = P.p[1], tz = P.p[2];
  G dp[3] = {G(), G(), G()};
  G dmu[3] = {G(), G(), G()};
  // opacity = sigmoid(logit)
  o.op += dop * P.o * (1 - P.o);
  // colour
  int K = (g->sh_degree + 1) * (g->sh_degree + 1);
  double Y[16], dY[48];
  sh_eval(g->sh_degree, P.dir, Y, dY);
  const double* sh = g->sh + (size_t)i * K * 3;
  G ddir[3] = {G(), G(), G()};
  for (int ch = 0; ch < 3; ++ch) {
    if (P.raw[ch] < 0) continue;
    for (int k = 0; k < K; ++k) {
      o.sh[k * 3 + ch] += dcol[ch] * Y[k];
      for (int a = 0; a < 3; ++a) ddir[a] += dcol[ch] * sh[k * 3 + ch] * dY[k * 3 + a];
    }
  }
  if constexpr (std::is_same<G, double>::value) sh_direction_error(g, cam, P, sh, K, dcol, ddir, Y, dY, o);
  G dd_dot = ddir[0] * P.dir[0] + ddir[1] * P.dir[1] + ddir[2] * P.dir[2];
  for (int a = 0; a < 3; ++a) dmu[a] += (ddir[a] - P.dir[a] * dd_dot) / P.vnorm;
  // depth and projected centre
  dp[2] += dd;
  dp[0] += du * fx / tz;
  dp[2] += -du * fx * tx / (tz * tz);
  dp[1] += dv * fy / tz;
  dp[2] += -dv * fy * ty / (tz * tz);
  // conic = inverse(cov): dL/dcov = -M Gm M (symmetric trace form)
  double M[4] = {P.conic[0], P.conic[1], P.conic[1], P.conic[2]};
  G Gm[4] = {dA, 0.5 * dB, 0.5 * dB, dC};
  G t1[4], Gs[4];
  matmul(M, Gm, t1, 2, 2, 2);
  matmul(t1, M, Gs, 2, 2, 2);
  for (G& x : Gs) x = -x;
  // cov = T S3 T^T + 0.3 I
  G GsT[6], H[9];
  double Tt[6];
  matmul(Gs, P.T, GsT, 2, 2, 3);
  transpose(P.T, Tt, 2, 3);
  matmul(Tt, GsT, H, 3, 2, 3);          // dL/dS3 = T^T Gs T
  G dT[6];
  matmul(GsT, P.S3, dT, 2, 3, 3);       // dL/dT = 2 Gs T S3
  for (G& x : dT) x *= 2;
  double Wt[9];
  G dJ[6];
  transpose(cam->R, Wt, 3, 3);
  matmul(dT, Wt, dJ, 2, 3, 3);          // T = J W
  dp[2] += dJ[0] * (-fx / (tz * tz)) + dJ[4] * (-fy / (tz * tz));
  if (!P.clampx) {
    dp[0] += dJ[2] * (-fx / (tz * tz));
    dp[2] += dJ[2] * (2 * fx * tx / (tz * tz * tz));
  } else {
    double xc = std::min(P.limx, std::max(-P.limx, P.xr));
    dp[2] += dJ[2] * (fx * xc / (tz * tz));
  }
  if (!P.clampy) {
    dp[1] += dJ[5] * (-fy / (tz * tz));
    dp[2] += dJ[5] * (2 * fy * ty / (tz * tz * tz));
  } else {
    double yc = std::min(P.limy, std::max(-P.limy, P.yr));
    dp[2] += dJ[5] * (fy * yc / (tz * tz));
  }
  // p = W mu + t
  for (int a = 0; a < 3; ++a) dmu[a] += cam->R[0 * 3 + a] * dp[0] + cam->R[1 * 3 + a] * dp[1] + cam->R[2 * 3 + a] * dp[2];
  for (int a = 0; a < 3; ++a) o.mu[a] += dmu[a];
  // S3 = Rq diag(s^2) Rq^T
  G RtH[9], RtHR[9];
  double Rqt[9];
  transpose(P.Rq, Rqt, 3, 3);
  matmul(Rqt, H, RtH, 3, 3, 3);
  matmul(RtH, P.Rq, RtHR, 3, 3, 3);
  for (int k = 0; k < 3; ++k) o.ls[k] += 2 * P.s[k] * RtHR[k * 4] * P.s[k];
  G dR[9], HR[9];
  matmul(H, P.Rq, HR, 3, 3, 3);
  for (int a = 0; a < 3; ++a)
    for (int k = 0; k < 3; ++k) dR[a * 3 + k] = 2 * HR[a * 3 + k] * P.s[k] * P.s[k];
  G dqn[4];
  rot_backward(P.qn, dR, dqn);
  G dot = dqn[0] * P.qn[0] + dqn[1] * P.qn[1] + dqn[2] * P.qn[2] + dqn[3] * P.qn[3];
  for (int k = 0; k < 4; ++k) o.q[k] += (dqn[k] - P.qn[k] * dot) / P.qnorm;
  if constexpr (std::is_same<G, double>::value)
    o.stat = std::sqrt(dmu[0] * dmu[0] + dmu[1] * dmu[1] + dmu[2] * dmu[2]);
}

void gaussian_backward(const orc_gaussians* g, const orc_camera* cam, const Proj& P, int64_t i,
                       const double* g2, const double* g2abs, orc_grads* out) {
  ParamGradT<double> o;
  gaussian_backward_local(g, cam, P, i, g2, o);
  const int K = (g->sh_degree + 1) * (g->sh_degree + 1);
  for (int a = 0; a < 3; ++a) out->means[3 * i + a] += o.mu[a];
  for (int k = 0; k < 3; ++k) out->log_scales[3 * i + k] += o.ls[k];
  for (int k = 0; k < 4; ++k) out->quats[4 * i + k] += o.q[k];
  out->opacity_logit[i] += o.op;
  for (int k = 0; k < K * 3; ++k) out->sh[(size_t)i * K * 3 + k] += o.sh[k];
  if (out->grad_stat) out->grad_stat[i] += o.stat;
  if (!g2abs || !out->scale_means) return;
  // Error scale of each parameter element: the same chain rule in running-error
  // arithmetic, fed per screen-space component the sum of |per-pixel term| times the
  // relative error that term may carry in float32.  Cancellation in the exact sums or
  // in the chain rule does not shrink it.
  AbsVal in[10];
  for (int j = 0; j < 10; ++j) in[j].v = g2abs[j];
  ParamGradT<AbsVal> c;
  gaussian_backward_local(g, cam, P, i, in, c);
  for (int a = 0; a < 3; ++a) out->scale_means[3 * i + a] += c.mu[a].v;
  for (int k = 0; k < 3; ++k) out->scale_log_scales[3 * i + k] += c.ls[k].v;
  for (int k = 0; k < 4; ++k) out->scale_quats[4 * i + k] += c.q[k].v;
  out->scale_opacity_logit[i] += c.op.v;
  for (int k = 0; k < K * 3; ++k) out->scale_sh[(size_t)i * K * 3 + k] += c.sh[k].v + o.xsh[k];
  for (int a = 0; a < 3; ++a) out->scale_means[3 * i + a] += o.xmu[a];
}

// ---------- 2-Wasserstein helpers (Eq. 7-9) ----------
void cov_of(const double* q, const double* s, double* S) {
  double n = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  double qn[4] = {q[0] / n, q[1] / n, q[2] / n, q[3] / n}, R[9];
  quat_to_rot(qn, R);
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double acc = 0;
      for (int k = 0; k < 3; ++k) acc += R[a * 3 + k] * s[k] * s[k] * R[b * 3 + k];
      S[a * 3 + b] = acc;
    }
}

// Optimal transport map from N(0,A) to N(0,B): A^-1/2 (A^1/2 B A^1/2)^1/2 A^-1/2.
void transport_map(const double* A, const double* B, double* Tm) {
  double Ah[9], Aih[9], t1[9], t2[9], mid[9];
  sym_fun(A, 0.5, Ah);
  sym_fun(A, -0.5, Aih);
  matmul(Ah, B, t1, 3, 3, 3);
  matmul(t1, Ah, t2, 3, 3, 3);
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) mid[a * 3 + b] = 0.5 * (t2[a * 3 + b] + t2[b * 3 + a]);
  double mh[9];
  sym_fun(mid, 0.5, mh);
  matmul(Aih, mh, t1, 3, 3, 3);
  matmul(t1, Aih, Tm, 3, 3, 3);
}

double w2_sq(const double* A, const double* B) {
  double Ah[9], t1[9], t2[9], mid[9], mh[9];
  sym_fun(A, 0.5, Ah);
  matmul(Ah, B, t1, 3, 3, 3);
  matmul(t1, Ah, t2, 3, 3, 3);
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) mid[a * 3 + b] = 0.5 * (t2[a * 3 + b] + t2[b * 3 + a]);
  sym_fun(mid, 0.5, mh);
  return A[0] + A[4] + A[8] + B[0] + B[4] + B[8] - 2 * (mh[0] + mh[4] + mh[8]);
}

void barycentre(const double* Si, const double* Sj, double* Sk) {
  double Tm[9], M[9], t1[9];
  transport_map(Si, Sj, Tm);
  for (int a = 0; a < 9; ++a) M[a] = 0.5 * ((a % 4 == 0 ? 1.0 : 0.0) + Tm[a]);
  matmul(M, Si, t1, 3, 3, 3);
  matmul(t1, M, Sk, 3, 3, 3);
  for (int a = 0; a < 3; ++a)
    for (int b = a + 1; b < 3; ++b) {
      double m = 0.5 * (Sk[a * 3 + b] + Sk[b * 3 + a]);
      Sk[a * 3 + b] = Sk[b * 3 + a] = m;
    }
}

// Rotation matrix -> unit quaternion (w >= 0).
void rot_to_quat(const double* R, double* q) {
  double tr = R[0] + R[4] + R[8];
  if (tr > 0) {
    double S = std::sqrt(tr + 1.0) * 2;
    q[0] = 0.25 * S; q[1] = (R[7] - R[5]) / S; q[2] = (R[2] - R[6]) / S; q[3] = (R[3] - R[1]) / S;
  } else if (R[0] > R[4] && R[0] > R[8]) {
    double S = std::sqrt(1.0 + R[0] - R[4] - R[8]) * 2;
    q[0] = (R[7] - R[5]) / S; q[1] = 0.25 * S; q[2] = (R[1] + R[3]) / S; q[3] = (R[2] + R[6]) / S;
  } else if (R[4] > R[8]) {
    double S = std::sqrt(1.0 + R[4] - R[0] - R[8]) * 2;
    q[0] = (R[2] - R[6]) / S; q[1] = (R[1] + R[3]) / S; q[2] = 0.25 * S; q[3] = (R[5] + R[7]) / S;
  } else {
    double S = std::sqrt(1.0 + R[8] - R[0] - R[4]) * 2;
    q[0] = (R[3] - R[1]) / S; q[1] = (R[2] + R[6]) / S; q[2] = (R[5] + R[7]) / S; q[3] = 0.25 * S;
  }
  if (q[0] < 0)
    for (int k = 0; k < 4; ++k) q[k] = -q[k];
}

// Covariance -> (unit quaternion, scales) by eigen-decomposition, scales descending.
void cov_to_qs(const double* S, double* q, double* s) {
  double w[3], V[9];
  eig_sym3(S, w, V);
  int ord[3] = {0, 1, 2};
  std::sort(ord, ord + 3, [&](int a, int b) { return w[a] > w[b]; });
  double R[9];
  for (int c = 0; c < 3; ++c)
    for (int r = 0; r < 3; ++r) R[r * 3 + c] = V[r * 3 + ord[c]];
  double det = R[0] * (R[4] * R[8] - R[5] * R[7]) - R[1] * (R[3] * R[8] - R[5] * R[6]) +
               R[2] * (R[3] * R[7] - R[4] * R[6]);
  if (det < 0)
    for (int r = 0; r < 3; ++r) R[r * 3 + 2] = -R[r * 3 + 2];
  rot_to_quat(R, q);
  for (int c = 0; c < 3; ++c) s[c] = std::sqrt(std::max(w[ord[c]], 0.0));
}

// Objective of Eq. 9 over theta = (q[4], s[3]) and its gradient.
double w2_objective(const double* th, const double* Si, const double* Sj, double* grad) {
  double Sk[9];
  cov_of(th, th + 4, Sk);
  double f = w2_sq(Sk, Si) + w2_sq(Sk, Sj);
  if (grad) {
    // d/dSk W2^2(Sk, B) = I - T_{Sk->B}
    double Ti[9], Tj[9], G[9];
    transport_map(Sk, Si, Ti);
    transport_map(Sk, Sj, Tj);
    for (int a = 0; a < 9; ++a) G[a] = 2 * (a % 4 == 0 ? 1.0 : 0.0) - Ti[a] - Tj[a];
    for (int a = 0; a < 3; ++a)
      for (int b = a + 1; b < 3; ++b) {
        double m = 0.5 * (G[a * 3 + b] + G[b * 3 + a]);
        G[a * 3 + b] = G[b * 3 + a] = m;
      }
    double n = std::sqrt(th[0] * th[0] + th[1] * th[1] + th[2] * th[2] + th[3] * th[3]);
    double qn[4] = {th[0] / n, th[1] / n, th[2] / n, th[3] / n}, R[9], Rt[9], t1[9], t2[9];
    quat_to_rot(qn, R);
    transpose(R, Rt, 3, 3);
    matmul(Rt, G, t1, 3, 3, 3);
    matmul(t1, R, t2, 3, 3, 3);
    const double* s = th + 4;
    for (int k = 0; k < 3; ++k) grad[4 + k] = 2 * s[k] * t2[k * 4];
    double GR[9], dR[9], dqn[4];
    matmul(G, R, GR, 3, 3, 3);
    for (int a = 0; a < 3; ++a)
      for (int k = 0; k < 3; ++k) dR[a * 3 + k] = 2 * GR[a * 3 + k] * s[k] * s[k];
    rot_backward(qn, dR, dqn);
    double dot = dqn[0] * qn[0] + dqn[1] * qn[1] + dqn[2] * qn[2] + dqn[3] * qn[3];
    for (int k = 0; k < 4; ++k) grad[k] = (dqn[k] - qn[k] * dot) / n;
  }
  return f;
}

}  // namespace

// =====================================================================================
extern "C" {

int orc_sh_basis(int32_t degree, const double dir[3], double* Y, double* dY) {
  if (degree < 0 || degree > 3) return -1;
  sh_eval(degree, dir, Y, dY);
  return 0;
}

int orc_project(const orc_gaussians* g, const orc_camera* cam, orc_projection* out) {
  if (!g || !cam || g->n < 0 || g->sh_degree < 0 || g->sh_degree > 3) return -1;
  std::vector<Proj> P = project_all(g, cam, nullptr, 0);
  for (int64_t i = 0; i < g->n; ++i) {
    const Proj& p = P[i];
    bool drawn = !p.culled;
    if (out->mean2d) { out->mean2d[2 * i] = drawn ? p.u : 0; out->mean2d[2 * i + 1] = drawn ? p.v : 0; }
    for (int k = 0; k < 3; ++k) {
      if (out->conic) out->conic[3 * i + k] = drawn ? p.conic[k] : 0;
      if (out->cov2d) out->cov2d[3 * i + k] = drawn ? p.cov[k] : 0;
      if (out->rgb) out->rgb[3 * i + k] = drawn ? p.rgb[k] : 0;
    }
    if (out->depth) out->depth[i] = p.p[2];
    if (out->opacity) out->opacity[i] = drawn ? p.o : 0;
    if (out->radius) out->radius[i] = drawn ? p.r : 0;
    if (out->rect)
      for (int k = 0; k < 4; ++k) out->rect[4 * i + k] = drawn ? p.rect[k] : (k < 2 ? 0 : -1);
    if (out->visible) out->visible[i] = p.visible ? 1 : 0;
  }
  return 0;
}

static int render_impl(const orc_gaussians* g, const orc_camera* cam, const orc_margins* mg,
                       const int32_t* tiles, int32_t n_tiles, double* rgb, double* depth, double* alpha,
                       double* T_final, int32_t* n_contrib, int32_t* n_eval, uint8_t* flags,
                       uint64_t* decision_hash, double* alt_rgb, double* alt_depth, double* alt_alpha,
                       int32_t* n_ties, int32_t n_threads) {
  if (!g || !cam || g->n < 0 || cam->width <= 0 || cam->height <= 0) return -1;
  std::vector<Proj> P = project_all(g, cam, mg, n_threads);
  std::vector<char> want = tile_mask(cam, tiles, n_tiles);
  auto bins = bin_tiles(P, cam, want, n_threads);
  int TX = tiles_x(cam), W = cam->width, H = cam->height;
  size_t HW = (size_t)W * H;
  const bool alt = alt_rgb || alt_depth || alt_alpha || n_ties;
  std::vector<uint64_t> tile_hash(bins.size(), 0);
  parallel_for((int64_t)bins.size(), n_threads, [&](int64_t t) {
    if (!want[t]) return;
    int x0 = (int)(t % TX) * kTile, y0 = (int)(t / TX) * kTile;
    uint64_t h = 0;
    std::vector<Tie> ties;
    for (int py = y0; py < std::min(H, y0 + kTile); ++py)
      for (int px = x0; px < std::min(W, x0 + kTile); ++px) {
        PixelResult R;
        ties.clear();
        blend_pixel(P, bins[t], px, py, mg, decision_hash != nullptr, R, nullptr, alt ? &ties : nullptr);
        size_t o = (size_t)py * W + px;
        for (int c = 0; c < 3; ++c) if (rgb) rgb[c * HW + o] = R.rgb[c];
        if (depth) depth[o] = R.depth;
        if (alpha) alpha[o] = 1 - R.T;
        if (T_final) T_final[o] = R.T;
        if (n_contrib) n_contrib[o] = R.n_contrib;
        if (n_eval) n_eval[o] = R.n_eval;
        if (flags) flags[o] = R.flags;
        if (alt) {
          // the other outcome of a single near-tie decision; none for two or more
          PixelResult A = R;
          if (ties.size() == 1) {
            A = PixelResult();
            blend_pixel_flipped(P, bins[t], px, py, mg, ties[0], A);
          }
          const double nan = std::nan("");
          const bool many = ties.size() > 1;
          for (int c = 0; c < 3; ++c) if (alt_rgb) alt_rgb[c * HW + o] = many ? nan : A.rgb[c];
          if (alt_depth) alt_depth[o] = many ? nan : A.depth;
          if (alt_alpha) alt_alpha[o] = many ? nan : 1 - A.T;
          if (n_ties) n_ties[o] = (int32_t)ties.size();
        }
        if (decision_hash) {
          h = mix(h, o);
          for (auto& c : R.contrib) h = mix(h, (uint64_t)c.g + 1);
          h = mix(h, (uint64_t)R.n_eval);
        }
      }
    tile_hash[t] = h;
  });
  if (decision_hash) {
    uint64_t h = 0;
    for (uint64_t x : tile_hash) h = mix(h, x);
    *decision_hash = h;
  }
  return 0;
}

int orc_render(const orc_gaussians* g, const orc_camera* cam, const orc_margins* mg,
               const int32_t* tiles, int32_t n_tiles, double* rgb, double* depth, double* alpha,
               double* T_final, int32_t* n_contrib, int32_t* n_eval, uint8_t* flags,
               uint64_t* decision_hash, int32_t n_threads) {
  return render_impl(g, cam, mg, tiles, n_tiles, rgb, depth, alpha, T_final, n_contrib, n_eval, flags,
                     decision_hash, nullptr, nullptr, nullptr, nullptr, n_threads);
}

int orc_render_outcomes(const orc_gaussians* g, const orc_camera* cam, const orc_margins* mg,
                        const int32_t* tiles, int32_t n_tiles, double* rgb, double* depth, double* alpha,
                        double* T_final, int32_t* n_contrib, uint8_t* flags, double* alt_rgb,
                        double* alt_depth, double* alt_alpha, int32_t* n_ties, int32_t n_threads) {
  if (!mg) return -1;
  return render_impl(g, cam, mg, tiles, n_tiles, rgb, depth, alpha, T_final, n_contrib, nullptr, flags,
                     nullptr, alt_rgb, alt_depth, alt_alpha, n_ties, n_threads);
}

int orc_render_bruteforce(const orc_gaussians* g, const orc_camera* cam, double* rgb, double* depth,
                          double* alpha) {
  if (!g || !cam || g->n < 0) return -1;
  std::vector<Proj> P = project_all(g, cam, nullptr, 1);
  int W = cam->width, H = cam->height;
  size_t HW = (size_t)W * H;
  for (int py = 0; py < H; ++py)
    for (int px = 0; px < W; ++px) {
      int tx = px / kTile, ty = py / kTile;
      std::vector<int> ids;
      for (int64_t i = 0; i < g->n; ++i)
        if (P[i].visible && in_rect(P[i].rect, tx, ty)) ids.push_back((int)i);
      std::sort(ids.begin(), ids.end(), [&](int a, int b) {
        float za = (float)P[a].p[2], zb = (float)P[b].p[2];
        return za < zb || (za == zb && a < b);
      });
      // C = sum_i c_i alpha_i prod_{j<i}(1 - alpha_j), written with explicit products.
      std::vector<double> al;
      std::vector<int> used;
      for (int id : ids) {
        double dx, dy, power = power_at(P[id], px, py, &dx, &dy);
        if (power > 0) continue;
        double a = std::min(kAlphaMax, P[id].o * std::exp(power));
        if (a < kAlphaMin) continue;
        al.push_back(a);
        used.push_back(id);
        double T = 1;
        for (double x : al) T *= (1 - x);
        if (T < kTStop) break;
      }
      double C[3] = {0, 0, 0}, D = 0, T = 1;
      for (size_t k = 0; k < used.size(); ++k) {
        double prod = 1;
        for (size_t j = 0; j < k; ++j) prod *= (1 - al[j]);
        for (int c = 0; c < 3; ++c) C[c] += P[used[k]].rgb[c] * al[k] * prod;
        D += P[used[k]].p[2] * al[k] * prod;
        T *= (1 - al[k]);
      }
      size_t o = (size_t)py * W + px;
      for (int c = 0; c < 3; ++c) rgb[c * HW + o] = C[c];
      depth[o] = D;
      alpha[o] = 1 - T;
    }
  return 0;
}

int orc_render_backward(const orc_gaussians* g, const orc_camera* cam, const orc_margins* mg,
                        const int32_t* tiles, int32_t n_tiles, const double* g_rgb,
                        const double* g_depth, const double* g_alpha, orc_grads* out,
                        int32_t n_threads) {
  if (!g || !cam || !out || g->n < 0) return -1;
  std::vector<Proj> P = project_all(g, cam, mg, n_threads);
  std::vector<char> want = tile_mask(cam, tiles, n_tiles);
  auto bins = bin_tiles(P, cam, want, n_threads);
  int TX = tiles_x(cam), W = cam->width, H = cam->height;
  size_t HW = (size_t)W * H;
  // Per (tile, list entry) screen-space gradients, reduced afterwards in tile order.
  std::vector<std::vector<double>> acc(bins.size()), accabs(bins.size());
  const bool scale = out->scale_means != nullptr;
  std::vector<std::vector<int32_t>> taint_lists(bins.size());
  parallel_for((int64_t)bins.size(), n_threads, [&](int64_t t) {
    if (!want[t] || bins[t].empty()) return;
    const auto& list = bins[t];
    std::vector<int32_t> slot(0);
    // map Gaussian -> entry slot within this tile
    std::vector<std::pair<int32_t, int32_t>> idx;
    idx.reserve(list.size());
    for (size_t k = 0; k < list.size(); ++k) idx.push_back({list[k].g, (int32_t)k});
    std::sort(idx.begin(), idx.end());
    auto slot_of = [&](int32_t gi) {
      auto it = std::lower_bound(idx.begin(), idx.end(), std::make_pair(gi, (int32_t)-1));
      return it->second;
    };
    acc[t].assign(list.size() * 10, 0.0);
    if (scale) accabs[t].assign(list.size() * 10, 0.0);
    int x0 = (int)(t % TX) * kTile, y0 = (int)(t / TX) * kTile;
    for (int py = y0; py < std::min(H, y0 + kTile); ++py)
      for (int px = x0; px < std::min(W, x0 + kTile); ++px) {
        size_t o = (size_t)py * W + px;
        PixelResult R;
        blend_pixel(P, list, px, py, mg, true, R);
        if (R.flags && out->taint)
          for (int32_t gi : R.touched) taint_lists[t].push_back(gi);
        double gC[3] = {g_rgb ? g_rgb[o] : 0, g_rgb ? g_rgb[HW + o] : 0, g_rgb ? g_rgb[2 * HW + o] : 0};
        double gD = g_depth ? g_depth[o] : 0, gA = g_alpha ? g_alpha[o] : 0;
        double S[3] = {0, 0, 0}, SD = 0, Tf = R.T;
        for (int k = (int)R.contrib.size() - 1; k >= 0; --k) {
          const Contribution& c = R.contrib[k];
          const Proj& p = P[c.g];
          double* a = &acc[t][(size_t)slot_of(c.g) * 10];
          double dummy[10];
          double* b = scale ? &accabs[t][(size_t)slot_of(c.g) * 10] : dummy;
          // relative error a float32 evaluation of this pixel's terms may carry: the alpha
          // margin of this contribution, the accumulated T margin of the pixel, and 32
          // units of 2^-24 for the rounding of the sums
          const double u = c.ma + R.t_err + 32.0 * kEps32;
          double w = c.alpha * c.Tb;
          for (int ch = 0; ch < 3; ++ch) a[6 + ch] += w * gC[ch];
          a[9] += w * gD;
          for (int ch = 0; ch < 3; ++ch) b[6 + ch] += u * std::fabs(w * gC[ch]);
          b[9] += u * std::fabs(w * gD);
          double dLda = 0;
          for (int ch = 0; ch < 3; ++ch) dLda += (p.rgb[ch] - S[ch]) * gC[ch];
          dLda += (p.p[2] - SD) * gD;
          dLda = c.Tb * dLda + gA * Tf / (1 - c.alpha);
          for (int ch = 0; ch < 3; ++ch) S[ch] = c.alpha * p.rgb[ch] + (1 - c.alpha) * S[ch];
          SD = c.alpha * p.p[2] + (1 - c.alpha) * SD;
          if (c.a <= kAlphaMax) {
            a[5] += dLda * c.G;
            double gp = dLda * c.a;  // dL/dpower
            a[2] += gp * (-0.5 * c.dx * c.dx);
            a[3] += gp * (-c.dx * c.dy);
            a[4] += gp * (-0.5 * c.dy * c.dy);
            a[0] += gp * (-p.conic[0] * c.dx - p.conic[1] * c.dy);
            a[1] += gp * (-p.conic[2] * c.dy - p.conic[1] * c.dx);
            b[5] += u * std::fabs(dLda * c.G);
            b[2] += u * std::fabs(gp * 0.5 * c.dx * c.dx);
            b[3] += u * std::fabs(gp * c.dx * c.dy);
            b[4] += u * std::fabs(gp * 0.5 * c.dy * c.dy);
            b[0] += u * std::fabs(gp) * (std::fabs(p.conic[0] * c.dx) + std::fabs(p.conic[1] * c.dy));
            b[1] += u * std::fabs(gp) * (std::fabs(p.conic[2] * c.dy) + std::fabs(p.conic[1] * c.dx));
          }
        }
      }
  });
  std::vector<double> g2((size_t)g->n * 10, 0.0), g2abs(scale ? (size_t)g->n * 10 : 0, 0.0);
  for (size_t t = 0; t < bins.size(); ++t) {
    if (acc[t].empty()) continue;
    for (size_t k = 0; k < bins[t].size(); ++k)
      for (int c = 0; c < 10; ++c) {
        g2[(size_t)bins[t][k].g * 10 + c] += acc[t][k * 10 + c];
        if (scale) g2abs[(size_t)bins[t][k].g * 10 + c] += accabs[t][k * 10 + c];
      }
    if (out->taint)
      for (int32_t gi : taint_lists[t]) out->taint[gi] = 1;
  }
  if (out->grad2d)
    for (size_t k = 0; k < g2.size(); ++k) out->grad2d[k] += g2[k];
  parallel_for((g->n + 1023) / 1024, n_threads, [&](int64_t b) {
    for (int64_t i = b * 1024; i < std::min<int64_t>(g->n, (b + 1) * 1024); ++i) {
      if (!P[i].visible) continue;
      if (out->vis_count) out->vis_count[i] += 1;
      gaussian_backward(g, cam, P[i], i, &g2[(size_t)i * 10], scale ? &g2abs[(size_t)i * 10] : nullptr, out);
    }
  });
  return 0;
}

// ---------------------------- voxel merge ----------------------------
int orc_voxel_keys(int64_t n, const double* means, double voxel, int32_t* keys) {
  if (n < 0 || !(voxel > 0)) return -1;
  float v = (float)voxel;
  for (int64_t i = 0; i < 3 * n; ++i) {
    float m = (float)means[i];
    float q = (float)((double)m / (double)v);  // the correctly rounded float32 quotient
    keys[i] = (int32_t)std::floor(q);
  }
  return 0;
}

int orc_covariance(const double q[4], const double s[3], double S[9]) {
  cov_of(q, s, S);
  return 0;
}

int orc_w2_barycentre(const double Si[9], const double Sj[9], double Sk[9]) {
  barycentre(Si, Sj, Sk);
  return 0;
}

double orc_w2_sq(const double A[9], const double B[9]) { return w2_sq(A, B); }

int orc_merge_mean(const double Si[9], const double mi[3], const double Sj[9], const double mj[3],
                   double mk[3]) {
  // Eq. 6: (Si^-1 + Sj^-1)^-1 (Si^-1 mi + Sj^-1 mj)
  double Pi[9], Pj[9], Ps[9], Psi[9], r[3];
  inv3(Si, Pi);
  inv3(Sj, Pj);
  for (int a = 0; a < 9; ++a) Ps[a] = Pi[a] + Pj[a];
  inv3(Ps, Psi);
  for (int a = 0; a < 3; ++a) {
    r[a] = 0;
    for (int b = 0; b < 3; ++b) r[a] += Pi[a * 3 + b] * mi[b] + Pj[a * 3 + b] * mj[b];
  }
  for (int a = 0; a < 3; ++a) {
    mk[a] = 0;
    for (int b = 0; b < 3; ++b) mk[a] += Psi[a * 3 + b] * r[b];
  }
  return 0;
}

int orc_w2_lbfgs(const double qi[4], const double si[3], const double qj[4], const double sj[3],
                 double t, const double delta[3], double qk[4], double sk[3], double Sk[9],
                 double* final_objective) {
  double Si[9], Sj[9];
  cov_of(qi, si, Si);
  cov_of(qj, sj, Sj);
  // Eq. 10: q0 = slerp(qi, qj, t) on the shorter arc, s0 = (si + sj)/2 + delta.
  double a[4], b[4];
  double na = std::sqrt(qi[0] * qi[0] + qi[1] * qi[1] + qi[2] * qi[2] + qi[3] * qi[3]);
  double nb = std::sqrt(qj[0] * qj[0] + qj[1] * qj[1] + qj[2] * qj[2] + qj[3] * qj[3]);
  for (int k = 0; k < 4; ++k) { a[k] = qi[k] / na; b[k] = qj[k] / nb; }
  double d = a[0] * b[0] + a[1] * b[1] + a[2] * b[2] + a[3] * b[3];
  if (d < 0) { for (double& x : b) x = -x; d = -d; }
  double th[7];
  if (d > 1 - 1e-12) {
    for (int k = 0; k < 4; ++k) th[k] = (1 - t) * a[k] + t * b[k];
  } else {
    double om = std::acos(std::min(1.0, d));
    double ca = std::sin((1 - t) * om) / std::sin(om), cb = std::sin(t * om) / std::sin(om);
    for (int k = 0; k < 4; ++k) th[k] = ca * a[k] + cb * b[k];
  }
  for (int k = 0; k < 3; ++k) th[4 + k] = 0.5 * (si[k] + sj[k]) + delta[k];
  // L-BFGS, memory 8, backtracking Armijo line search.
  const int m = 8, D = 7;
  std::vector<std::vector<double>> S, Yv;
  std::vector<double> rho;
  double gcur[7], gnew[7], dir[7], xnew[7];
  double f = w2_objective(th, Si, Sj, gcur);
  int it = 0;
  for (; it < 5000; ++it) {
    double gn = 0;
    for (double x : gcur) gn += x * x;
    if (std::sqrt(gn) < 1e-15) break;
    // two-loop recursion
    double q[7];
    std::memcpy(q, gcur, sizeof(q));
    std::vector<double> al(S.size());
    for (int k = (int)S.size() - 1; k >= 0; --k) {
      double s = 0;
      for (int c = 0; c < D; ++c) s += S[k][c] * q[c];
      al[k] = rho[k] * s;
      for (int c = 0; c < D; ++c) q[c] -= al[k] * Yv[k][c];
    }
    double gamma = 1.0;
    if (!S.empty()) {
      double sy = 0, yy = 0;
      for (int c = 0; c < D; ++c) { sy += S.back()[c] * Yv.back()[c]; yy += Yv.back()[c] * Yv.back()[c]; }
      gamma = sy / yy;
    } else {
      gamma = 1e-3 / std::max(1e-300, std::sqrt(gn));
    }
    for (int c = 0; c < D; ++c) q[c] *= gamma;
    for (size_t k = 0; k < S.size(); ++k) {
      double yq = 0;
      for (int c = 0; c < D; ++c) yq += Yv[k][c] * q[c];
      double beta = rho[k] * yq;
      for (int c = 0; c < D; ++c) q[c] += S[k][c] * (al[k] - beta);
    }
    for (int c = 0; c < D; ++c) dir[c] = -q[c];
    double slope = 0;
    for (int c = 0; c < D; ++c) slope += dir[c] * gcur[c];
    if (slope >= 0) {  // not a descent direction: restart from steepest descent
      S.clear(); Yv.clear(); rho.clear();
      for (int c = 0; c < D; ++c) dir[c] = -gcur[c] * 1e-3 / std::sqrt(gn);
      slope = 0;
      for (int c = 0; c < D; ++c) slope += dir[c] * gcur[c];
    }
    double step = 1.0, fnew = 0;
    bool ok = false;
    for (int ls = 0; ls < 60; ++ls) {
      for (int c = 0; c < D; ++c) xnew[c] = th[c] + step * dir[c];
      fnew = w2_objective(xnew, Si, Sj, gnew);
      if (fnew <= f + 1e-4 * step * slope) { ok = true; break; }
      step *= 0.5;
    }
    if (!ok) break;
    std::vector<double> sv(D), yv(D);
    double sy = 0;
    for (int c = 0; c < D; ++c) { sv[c] = xnew[c] - th[c]; yv[c] = gnew[c] - gcur[c]; sy += sv[c] * yv[c]; }
    if (sy > 1e-300) {
      S.push_back(sv); Yv.push_back(yv); rho.push_back(1.0 / sy);
      if ((int)S.size() > m) { S.erase(S.begin()); Yv.erase(Yv.begin()); rho.erase(rho.begin()); }
    }
    std::memcpy(th, xnew, sizeof(th));
    std::memcpy(gcur, gnew, sizeof(gcur));
    if (f - fnew <= 1e-18 * std::max(1e-300, std::fabs(f)) && f - fnew >= 0 && it > 50) { f = fnew; break; }
    f = fnew;
  }
  double n = std::sqrt(th[0] * th[0] + th[1] * th[1] + th[2] * th[2] + th[3] * th[3]);
  for (int k = 0; k < 4; ++k) qk[k] = th[k] / n;
  for (int k = 0; k < 3; ++k) sk[k] = std::fabs(th[4 + k]);
  cov_of(qk, sk, Sk);
  if (final_objective) *final_objective = f;
  return it;
}

int orc_voxel_merge(const orc_gaussians* g, const uint64_t* birth, double voxel,
                    const orc_merge_params* p, double* out_means, double* out_log_scales,
                    double* out_quats, double* out_opacity_logit, double* out_sh,
                    uint64_t* out_birth, double* out_cov, int32_t* partner, int64_t* n_out,
                    double tie_rel, uint8_t* tie_flag) {
  if (!g || !birth || !p || g->n < 0 || !(voxel > 0)) return -1;
  int64_t n = g->n;
  int K = (g->sh_degree + 1) * (g->sh_degree + 1);
  std::vector<int32_t> keys((size_t)3 * n);
  orc_voxel_keys(n, g->means, voxel, keys.data());
  // Eq. 3 mask
  std::vector<char> elig(n, 1);
  for (int64_t i = 0; i < n; ++i) {
    bool ok = true;
    if (p->grad_stat) {
      double gs = p->grad_stat[i];  // Eq. 3: mean gradient norm over the views that drew it
      if (p->vis_count) gs = p->vis_count[i] > 0 ? (double)(float)(gs / p->vis_count[i]) : 0.0;
      ok = ok && gs < p->grad_tau;
    }
    if (p->kf_id) ok = ok && p->kf_id[i] >= p->kf_min && p->kf_id[i] <= p->kf_max;
    elig[i] = ok;
  }
  // voxel -> members
  std::map<std::tuple<int, int, int>, std::vector<int64_t>> vox;
  for (int64_t i = 0; i < n; ++i)
    if (elig[i]) vox[{keys[3 * i], keys[3 * i + 1], keys[3 * i + 2]}].push_back(i);
  std::vector<double> cov((size_t)9 * n), prec((size_t)9 * n);
  for (int64_t i = 0; i < n; ++i) {
    double s[3];
    for (int k = 0; k < 3; ++k) s[k] = std::exp(g->log_scales[3 * i + k]);
    cov_of(g->quats + 4 * i, s, &cov[9 * i]);
    inv3(&cov[9 * i], &prec[9 * i]);
  }
  std::vector<int64_t> part(n, -1);
  if (tie_flag) std::memset(tie_flag, 0, (size_t)n);
  struct Cand { double d2; uint64_t bi, bj; int64_t i, j; };
  for (auto& kv : vox) {
    auto mem = kv.second;
    if (mem.size() < 2) continue;
    std::sort(mem.begin(), mem.end(), [&](int64_t a, int64_t b) {
      return birth[a] < birth[b] || (birth[a] == birth[b] && a < b);
    });
    std::vector<Cand> cands;
    for (size_t a = 0; a < mem.size(); ++a)
      for (size_t b = a + 1; b < mem.size(); ++b) {
        int64_t i = mem[a], j = mem[b];  // i older than j
        double d[3], d2 = 0;
        for (int k = 0; k < 3; ++k) d[k] = g->means[3 * j + k] - g->means[3 * i + k];
        for (int r = 0; r < 3; ++r)
          for (int c = 0; c < 3; ++c) d2 += d[r] * prec[9 * i + r * 3 + c] * d[c];  // Eq. 4
        if (tie_flag && std::fabs(d2 - p->chi2) < tie_rel * p->chi2) tie_flag[i] = tie_flag[j] = 1;
        if (d2 < p->chi2) cands.push_back({d2, birth[i], birth[j], i, j});
      }
    std::sort(cands.begin(), cands.end(), [](const Cand& x, const Cand& y) {
      return std::tie(x.d2, x.bi, x.bj, x.i, x.j) < std::tie(y.d2, y.bi, y.bj, y.i, y.j);
    });
    // The greedy outcome depends only on the order of candidates that share a member.
    if (tie_flag)
      for (size_t k = 0; k < cands.size(); ++k)
        for (size_t l = k + 1; l < cands.size() && cands[l].d2 - cands[k].d2 <= tie_rel * cands[l].d2; ++l) {
          const Cand &x = cands[k], &y = cands[l];
          if (x.i == y.i || x.i == y.j || x.j == y.i || x.j == y.j)
            tie_flag[x.i] = tie_flag[x.j] = tie_flag[y.i] = tie_flag[y.j] = 1;
        }
    for (const Cand& c : cands) {
      if (part[c.i] >= 0 || part[c.j] >= 0) continue;
      part[c.i] = c.j;
      part[c.j] = c.i;
      if (!p->greedy) break;
    }
  }
  int64_t w = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (partner) partner[i] = (int32_t)part[i];
    bool dropped = part[i] >= 0 && (birth[part[i]] < birth[i] || (birth[part[i]] == birth[i] && part[i] < i));
    if (dropped) continue;
    int64_t j = part[i];
    double Sk[9];
    if (j >= 0) {
      orc_merge_mean(&cov[9 * i], g->means + 3 * i, &cov[9 * j], g->means + 3 * j, out_means + 3 * w);
      barycentre(&cov[9 * i], &cov[9 * j], Sk);
      double q[4], s[3];
      cov_to_qs(Sk, q, s);
      for (int k = 0; k < 4; ++k) out_quats[4 * w + k] = q[k];
      for (int k = 0; k < 3; ++k) out_log_scales[3 * w + k] = std::log(s[k]);
    } else {
      std::memcpy(Sk, &cov[9 * i], sizeof(Sk));
      for (int k = 0; k < 3; ++k) out_means[3 * w + k] = g->means[3 * i + k];
      for (int k = 0; k < 4; ++k) out_quats[4 * w + k] = g->quats[4 * i + k];
      for (int k = 0; k < 3; ++k) out_log_scales[3 * w + k] = g->log_scales[3 * i + k];
    }
    out_opacity_logit[w] = g->opacity_logit[i];
    std::memcpy(out_sh + (size_t)w * K * 3, g->sh + (size_t)i * K * 3, sizeof(double) * K * 3);
    out_birth[w] = birth[i];
    if (out_cov) {
      const int idx[6] = {0, 1, 2, 4, 5, 8};
      for (int k = 0; k < 6; ++k) out_cov[6 * w + k] = Sk[idx[k]];
    }
    ++w;
  }
  *n_out = w;
  return 0;
}

int orc_adam(int64_t n, double* param, const double* grad, double* m, double* v, double lr,
             double b1, double b2, double eps, int32_t step) {
  if (n < 0 || step < 1) return -1;
  double c1 = 1 - std::pow(b1, step), c2 = 1 - std::pow(b2, step);
  for (int64_t i = 0; i < n; ++i) {
    m[i] = b1 * m[i] + (1 - b1) * grad[i];
    v[i] = b2 * v[i] + (1 - b2) * grad[i] * grad[i];
    double mh = m[i] / c1, vh = v[i] / c2;
    param[i] -= lr * mh / (std::sqrt(vh) + eps);
  }
  return 0;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Mapping loss, Eq. 12.  SSIM (Wang et al.) with an 11x11 Gaussian window of standard
// deviation 1.5 (normalised to sum 1), constants (0.01)^2 and (0.03)^2 for values in
// [0, 1], evaluated at every pixel with the window cut by the image border (zero
// padding).  Written as plain windowed sums; the gradient goes through the three window
// moments of x (mean, mean of x^2, mean of x*y) that SSIM depends on.
namespace {
constexpr int kWin = 11, kHalf = 5;
constexpr double kSigma = 1.5, kC1 = 0.01 * 0.01, kC2 = 0.03 * 0.03;

void ssim_window(double w[kWin]) {
  double sum = 0;
  for (int i = 0; i < kWin; ++i) {
    double t = i - kHalf;
    w[i] = std::exp(-t * t / (2 * kSigma * kSigma));
    sum += w[i];
  }
  for (int i = 0; i < kWin; ++i) w[i] /= sum;
}
}  // namespace

int orc_mapping_loss(int32_t n_views, int32_t H, int32_t W, const double* x, const double* y,
                     const double* d, const double* dt, double lambda, double w_depth,
                     double* loss, double* g_rgb, double* g_depth) {
  if (n_views < 0 || H <= 0 || W <= 0 || !x || !y || !loss) return -1;
  double w1[kWin];
  ssim_window(w1);
  const int64_t HW = (int64_t)H * W;
  std::vector<double> d1(HW), d2(HW), d3(HW);  // dS/dm1, dS/dm2, dS/dm3 per pixel
  for (int v = 0; v < n_views; ++v) {
    double l1 = 0, ssim_sum = 0, ld = 0;
    for (int c = 0; c < 3; ++c) {
      const double* X = x + ((int64_t)v * 3 + c) * HW;
      const double* Y = y + ((int64_t)v * 3 + c) * HW;
      double* G = g_rgb ? g_rgb + ((int64_t)v * 3 + c) * HW : nullptr;
      for (int64_t p = 0; p < HW; ++p) l1 += std::fabs(X[p] - Y[p]);
      for (int qy = 0; qy < H; ++qy)
        for (int qx = 0; qx < W; ++qx) {
          double mx = 0, my = 0, mxx = 0, myy = 0, mxy = 0;
          for (int a = -kHalf; a <= kHalf; ++a)
            for (int b = -kHalf; b <= kHalf; ++b) {
              int py = qy + a, px = qx + b;
              if (py < 0 || py >= H || px < 0 || px >= W) continue;  // zero padding
              double wt = w1[a + kHalf] * w1[b + kHalf];
              double xv = X[(int64_t)py * W + px], yv = Y[(int64_t)py * W + px];
              mx += wt * xv; my += wt * yv;
              mxx += wt * xv * xv; myy += wt * yv * yv; mxy += wt * xv * yv;
            }
          double sx = mxx - mx * mx, sy = myy - my * my, sxy = mxy - mx * my;
          double A1 = 2 * mx * my + kC1, A2 = 2 * sxy + kC2;
          double B1 = mx * mx + my * my + kC1, B2 = sx + sy + kC2;
          double S = A1 * A2 / (B1 * B2);
          ssim_sum += S;
          // dS w.r.t. mu_x, sigma_x^2, sigma_xy, then to the moments m1 = E[x], m2 = E[x^2], m3 = E[xy]
          double dmu = 2 * my * A2 / (B1 * B2) - S * 2 * mx / B1;
          double dsx = -S / B2;
          double dsxy = 2 * A1 / (B1 * B2);
          int64_t q = (int64_t)qy * W + qx;
          d1[q] = dmu + dsx * (-2 * mx) + dsxy * (-my);
          d2[q] = dsx;
          d3[q] = dsxy;
        }
      if (G) {
        const double n = 3.0 * (double)HW;
        for (int py = 0; py < H; ++py)
          for (int px = 0; px < W; ++px) {
            double a1 = 0, a2 = 0, a3 = 0;
            for (int a = -kHalf; a <= kHalf; ++a)
              for (int b = -kHalf; b <= kHalf; ++b) {
                int qy = py + a, qx = px + b;
                if (qy < 0 || qy >= H || qx < 0 || qx >= W) continue;  // windows exist at image pixels only
                double wt = w1[a + kHalf] * w1[b + kHalf];
                int64_t q = (int64_t)qy * W + qx;
                a1 += wt * d1[q]; a2 += wt * d2[q]; a3 += wt * d3[q];
              }
            int64_t p = (int64_t)py * W + px;
            double dssim = (a1 + 2 * X[p] * a2 + Y[p] * a3) / n;
            double diff = X[p] - Y[p];
            double sgn = diff > 0 ? 1.0 : (diff < 0 ? -1.0 : 0.0);
            G[p] = (1 - lambda) * sgn / n - lambda * dssim;
          }
      }
    }
    if (dt && d) {
      const double* D = d + (int64_t)v * HW;
      const double* Dt = dt + (int64_t)v * HW;
      double* GD = g_depth ? g_depth + (int64_t)v * HW : nullptr;
      for (int64_t p = 0; p < HW; ++p) {
        bool valid = Dt[p] > 0;
        double diff = D[p] - Dt[p];
        if (valid) ld += std::fabs(diff);
        if (GD) GD[p] = valid ? w_depth * (diff > 0 ? 1.0 : (diff < 0 ? -1.0 : 0.0)) / (double)HW : 0.0;
      }
    } else if (g_depth) {
      for (int64_t p = 0; p < HW; ++p) g_depth[(int64_t)v * HW + p] = 0;
    }
    loss[3 * v] = (1 - lambda) * l1 / (3.0 * (double)HW);
    loss[3 * v + 1] = lambda * (1 - ssim_sum / (3.0 * (double)HW));
    loss[3 * v + 2] = w_depth * ld / (double)HW;
  }
  return 0;
}

int orc_iso_loss(int64_t n, const double* log_scales, double w_iso, double* loss, double* grad_ls) {
  if (n < 0 || !loss) return -1;
  double acc = 0;
  const double scale = n > 0 ? w_iso / (3.0 * (double)n) : 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double s[3], mean = 0;
    for (int k = 0; k < 3; ++k) { s[k] = std::exp(log_scales[3 * i + k]); mean += s[k] / 3; }
    double sg[3], sgsum = 0;
    for (int k = 0; k < 3; ++k) {
      double dlt = s[k] - mean;
      acc += std::fabs(dlt);
      sg[k] = dlt > 0 ? 1.0 : (dlt < 0 ? -1.0 : 0.0);
      sgsum += sg[k];
    }
    if (grad_ls)
      for (int k = 0; k < 3; ++k)  // d|s_k - mean|/ds_j summed over k, times ds_j/dlog s_j = s_j
        grad_ls[3 * i + k] += scale * (sg[k] - sgsum / 3) * s[k];
  }
  *loss = scale * acc;
  return 0;
}

// ---------------------------------------------------------------------------
// Patch-Grid sampling (Sec. II-B): densify patches with too few keypoints.
int orc_patch_grid(const orc_camera* cam, int32_t n_kp, const float* kp_uv, const float* kp_depth,
                   const float* depth_image, int32_t patch, int32_t min_keypoints, int32_t grid,
                   double* out, int32_t* source, int64_t* n_out) {
  if (!cam || !out || !n_out || n_kp < 0 || (n_kp > 0 && !kp_uv) || patch <= 0 || grid <= 0) return -1;
  const int W = cam->width, H = cam->height;
  const int PX = (W + patch - 1) / patch, PY = (H + patch - 1) / patch;
  std::vector<int> count((size_t)PX * PY, 0);
  for (int k = 0; k < n_kp; ++k) {
    float u = kp_uv[2 * k], v = kp_uv[2 * k + 1];
    if (!(u >= 0 && u < W && v >= 0 && v < H)) continue;
    count[(size_t)((int)v / patch) * PX + (int)u / patch] += 1;
  }
  int64_t n = 0;
  for (int py = 0; py < PY; ++py)
    for (int px = 0; px < PX; ++px) {
      if (count[(size_t)py * PX + px] >= min_keypoints) continue;
      // the patch as clipped by the image
      const double x0 = (double)px * patch, y0 = (double)py * patch;
      const double pw = std::min<double>(patch, W - x0), ph = std::min<double>(patch, H - y0);
      for (int a = 0; a < grid; ++a)
        for (int b = 0; b < grid; ++b) {
          const float u = (float)(x0 + (b + 0.5) * pw / grid), v = (float)(y0 + (a + 0.5) * ph / grid);
          double d = -1;
          int src = 0;
          if (depth_image) {
            float di = depth_image[(size_t)(int)v * W + (int)u];
            if (di > 0) d = di;
          }
          if (!(d > 0) && kp_depth) {
            int best = -1;
            float bd = 0;
            for (int k = 0; k < n_kp; ++k) {
              if (!(kp_depth[k] > 0)) continue;
              float du = kp_uv[2 * k] - u, dv = kp_uv[2 * k + 1] - v;
              float du2 = du * du, dv2 = dv * dv;
              float d2 = du2 + dv2;  // float32, as written (built without contraction)
              if (best < 0 || d2 < bd) { best = k; bd = d2; }
            }
            if (best >= 0) { d = kp_depth[best]; src = 1; }
          }
          if (!(d > 0)) continue;
          const double xc = ((double)u - cam->cx) / cam->fx * d, yc = ((double)v - cam->cy) / cam->fy * d;
          const double pc[3] = {xc - cam->t[0], yc - cam->t[1], d - cam->t[2]};
          double* o = out + 6 * n;
          o[0] = u; o[1] = v; o[2] = d;
          for (int r = 0; r < 3; ++r)
            o[3 + r] = cam->R[0 * 3 + r] * pc[0] + cam->R[1 * 3 + r] * pc[1] + cam->R[2 * 3 + r] * pc[2];
          if (source) source[n] = src;
          ++n;
        }
    }
  *n_out = n;
  return 0;
}
