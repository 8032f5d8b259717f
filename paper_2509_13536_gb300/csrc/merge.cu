// Voxel-space merge of geometrically similar Gaussians (Sec. II-D), sm_103a.
//
//  1. k_voxel_prep   Eq. 3 mask, voxel coordinates floor(mu/v) (IEEE f32 quotient),
//                    bounding box of the occupied voxels.
//  2. k_voxel_pack   voxel coordinates packed relative to the box into one u32 key
//                    (ineligible Gaussians get the all-ones key and sort last).
//  3. radix sort of (key, index); segment heads -> one (start, end) per voxel with two
//                    or more members (a single member has no pair).
//  4. k_voxel_pairs  8 lanes per voxel of <= 8 members, a whole warp per voxel of
//                    9..32, a block per voxel of 33..256 (members in shared
//                    memory) or of more (members in global scratch): members ranked by
//                    (birth, index), Eq. 4 for every older/younger pair, greedy
//                    disjoint pairing on (d2, birth_i, birth_j, i, j) below chi2,
//                    then the merge of each accepted pair: Eq. 6 mean, the
//                    equal-weight 2-Wasserstein barycentre (minimiser of Eq. 9) in
//                    closed form, eigen-decomposition back to (quaternion, scales).
//  5. ordered compaction: survivors keep input order, merged values in G_i's slot.
#include <cstring>

#include "internal.h"

namespace mgs {

struct MergeWs {
  int32_t* vox;            // [n][3] voxel coordinates of eligible Gaussians
  uint32_t* keys[2];       // [n]
  uint32_t* perm[2];       // [n]
  uint32_t* flags;         // [n] segment heads, then keep flags
  uint32_t* pos;           // [n] exclusive scans
  uint2* segs;             // [n] (first, end) in perm of each voxel with >= 2 members
  uint32_t tsize;          // hash table slots: a power of two >= 2n
  uint32_t* tkey;          // [tsize] voxel key of each slot (kNoKey: empty)
  uint32_t* tcount;        // [tsize] members per slot
  uint32_t* toff;          // [tsize] first position of each slot's members in perm
  uint32_t* tscratch;      // scan scratch over the table
  int32_t* partner;        // [n]
  float* mmean;            // [n][3] merged mean (valid where the Gaussian survives a merge)
  float* mquat;            // [n][4]
  float* mlogs;            // [n][3]
  uint32_t* big;           // [n] voxel ids with more than 32 members
  uint32_t* huge;          // [n] voxel ids with more than 256 members
  // members of the huge voxels, ranked by (birth, index), at their voxel's positions of
  // the sorted order
  int64_t* h_idx;          // [n]
  float* h_mu;             // [n][3]
  float* h_P;              // [n][6] precision (inverse covariance)
  int32_t* h_match;        // [n]
  uint2* pairs;            // [n/2 + 1] accepted (older, younger) pairs
  int32_t* hdr;            // 16 ints: bbox min xyz, max xyz, n_elig, err, n_vox, n_big, n_out, n_pairs,
                           // L-BFGS iterations (2 ints), n_huge
  uint32_t* scratch;       // sort / scan scratch
};

namespace {

constexpr int kWarpVoxel = 32;
constexpr int kBlockVoxel = 256;
constexpr int64_t kPersistBlocks = 152 * 8;  // grid of the grid-stride kernels: 8 blocks per SM
constexpr uint32_t kNoKey = 0xffffffffu;

__device__ __forceinline__ bool older(uint64_t ba, int64_t a, uint64_t bb, int64_t b) {
  return ba < bb || (ba == bb && a < b);
}

__device__ __forceinline__ void load_qs(const Geom& geo, int64_t i, float q[4], float s[3]) {
  for (int k = 0; k < 4; ++k) q[k] = ld_dt(geo.qs, geo.qdt, 4 * i + k);
  float n = rsqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  for (int k = 0; k < 4; ++k) q[k] *= n;
  for (int k = 0; k < 3; ++k) s[k] = expf(ld_dt(geo.ls, geo.dt, 3 * i + k));
}

// R diag(d) R^T as 6 unique entries xx xy xz yy yz zz
__device__ __forceinline__ void rdrt(const float R[9], const float d[3], float o[6]) {
  o[0] = R[0] * R[0] * d[0] + R[1] * R[1] * d[1] + R[2] * R[2] * d[2];
  o[1] = R[0] * R[3] * d[0] + R[1] * R[4] * d[1] + R[2] * R[5] * d[2];
  o[2] = R[0] * R[6] * d[0] + R[1] * R[7] * d[1] + R[2] * R[8] * d[2];
  o[3] = R[3] * R[3] * d[0] + R[4] * R[4] * d[1] + R[5] * R[5] * d[2];
  o[4] = R[3] * R[6] * d[0] + R[4] * R[7] * d[1] + R[5] * R[8] * d[2];
  o[5] = R[6] * R[6] * d[0] + R[7] * R[7] * d[1] + R[8] * R[8] * d[2];
}

__device__ __forceinline__ void precision_of(const Geom& geo, int64_t i, float P[6]) {
  float q[4], s[3], R[9];
  load_qs(geo, i, q, s);
  quat_rot(q, R);
  float d[3] = {1.f / (s[0] * s[0]), 1.f / (s[1] * s[1]), 1.f / (s[2] * s[2])};
  rdrt(R, d, P);
}

__device__ __forceinline__ float mahalanobis2(const float P[6], const float* mi, const float* mj) {
  float d0 = mj[0] - mi[0], d1 = mj[1] - mi[1], d2 = mj[2] - mi[2];
  return P[0] * d0 * d0 + P[3] * d1 * d1 + P[5] * d2 * d2 +
         2.f * (P[1] * d0 * d1 + P[2] * d0 * d2 + P[4] * d1 * d2);
}

// Cyclic Jacobi on a symmetric 3x3 (full row-major A), eigenvectors in the columns of V.
__device__ void jacobi3(float A[9], float V[9]) {
  for (int i = 0; i < 9; ++i) V[i] = (i % 4 == 0) ? 1.f : 0.f;
  const int P[3] = {0, 0, 1}, Q[3] = {1, 2, 2};
  for (int sweep = 0; sweep < 8; ++sweep) {
    float off = A[1] * A[1] + A[2] * A[2] + A[5] * A[5];
    float dia = A[0] * A[0] + A[4] * A[4] + A[8] * A[8];
    if (off <= 1e-14f * dia) break;
    for (int r = 0; r < 3; ++r) {
      int p = P[r], q = Q[r];
      float apq = A[3 * p + q];
      if (apq == 0.f) continue;
      float theta = (A[3 * q + q] - A[3 * p + p]) / (2.f * apq);
      float tt = copysignf(1.f, theta) / (fabsf(theta) + sqrtf(theta * theta + 1.f));
      float c = rsqrtf(tt * tt + 1.f), s = tt * c;
      for (int k = 0; k < 3; ++k) {
        float akp = A[3 * k + p], akq = A[3 * k + q];
        A[3 * k + p] = c * akp - s * akq;
        A[3 * k + q] = s * akp + c * akq;
      }
      for (int k = 0; k < 3; ++k) {
        float apk = A[3 * p + k], aqk = A[3 * q + k];
        A[3 * p + k] = c * apk - s * aqk;
        A[3 * q + k] = s * apk + c * aqk;
      }
      for (int k = 0; k < 3; ++k) {
        float vkp = V[3 * k + p], vkq = V[3 * k + q];
        V[3 * k + p] = c * vkp - s * vkq;
        V[3 * k + q] = s * vkp + c * vkq;
      }
    }
  }
}

// Unit quaternion (w >= 0) of a proper rotation matrix.
__device__ void rot_quat(const float R[9], float q[4]) {
  float tr = R[0] + R[4] + R[8];
  if (tr > 0.f) {
    float S = sqrtf(tr + 1.f) * 2.f;
    q[0] = 0.25f * S; q[1] = (R[7] - R[5]) / S; q[2] = (R[2] - R[6]) / S; q[3] = (R[3] - R[1]) / S;
  } else if (R[0] > R[4] && R[0] > R[8]) {
    float S = sqrtf(1.f + R[0] - R[4] - R[8]) * 2.f;
    q[0] = (R[7] - R[5]) / S; q[1] = 0.25f * S; q[2] = (R[1] + R[3]) / S; q[3] = (R[2] + R[6]) / S;
  } else if (R[4] > R[8]) {
    float S = sqrtf(1.f + R[4] - R[0] - R[8]) * 2.f;
    q[0] = (R[2] - R[6]) / S; q[1] = (R[1] + R[3]) / S; q[2] = 0.25f * S; q[3] = (R[5] + R[7]) / S;
  } else {
    float S = sqrtf(1.f + R[8] - R[0] - R[4]) * 2.f;
    q[0] = (R[3] - R[1]) / S; q[1] = (R[2] + R[6]) / S; q[2] = (R[5] + R[7]) / S; q[3] = 0.25f * S;
  }
  float n = rsqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  if (q[0] < 0.f) n = -n;
  for (int k = 0; k < 4; ++k) q[k] *= n;
}

// ---- Eq. 9 by the paper's solver: L-BFGS over (q, s) from the Eq. 10 start ----------
// Objective W2^2(Sk, A) + W2^2(Sk, B) with Sk = R(q/|q|) diag(s^2) R^T, all in the
// frame of Sigma_i.  W2^2(Sk, X) = tr Sk + tr X - 2 tr (Sk^1/2 X Sk^1/2)^1/2 (Eq. 8) and
// dW2^2/dSk = I - T, T = Sk^-1/2 (Sk^1/2 X Sk^1/2)^1/2 Sk^-1/2 (the transport map).
constexpr int kLbfgsMem = 6, kLbfgsIters = 200;

// C = H X H for symmetric H, X (row-major 3x3), result symmetrised
__device__ __forceinline__ void sandwich(const float H[9], const float X[9], float C[9]) {
  float t[9];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) t[3 * a + b] = H[3 * a] * X[b] + H[3 * a + 1] * X[3 + b] + H[3 * a + 2] * X[6 + b];
  for (int a = 0; a < 3; ++a)
    for (int b = a; b < 3; ++b) {
      const float x = t[3 * a] * H[b] + t[3 * a + 1] * H[3 + b] + t[3 * a + 2] * H[6 + b];
      C[3 * a + b] = x;
      C[3 * b + a] = x;
    }
}

__device__ __forceinline__ void rdrt9(const float R[9], const float d[3], float o[9]) {
  float u[6];
  rdrt(R, d, u);
  o[0] = u[0]; o[1] = u[1]; o[2] = u[2]; o[3] = u[1]; o[4] = u[3]; o[5] = u[4]; o[6] = u[2]; o[7] = u[4]; o[8] = u[5];
}

// f(th) and its gradient; th = (q[4], s[3]).  *gsig (optional): Frobenius norm of the
// gradient with respect to Sk itself, 2I - T_A - T_B, which vanishes only at the minimum.
__device__ float w2_objective(const float th[7], const float A[9], const float B[9], float g[7],
                              float* gsig = nullptr) {
  const float qn2 = th[0] * th[0] + th[1] * th[1] + th[2] * th[2] + th[3] * th[3];
  const float iq = rsqrtf(qn2);
  const float qn[4] = {th[0] * iq, th[1] * iq, th[2] * iq, th[3] * iq};
  float R[9];
  quat_rot(qn, R);
  const float s[3] = {th[4], th[5], th[6]};
  const float as[3] = {fabsf(s[0]), fabsf(s[1]), fabsf(s[2])};
  const float ias[3] = {1.f / as[0], 1.f / as[1], 1.f / as[2]};
  float Hh[9], Hi[9];  // Sk^1/2, Sk^-1/2
  rdrt9(R, as, Hh);
  rdrt9(R, ias, Hi);
  float f = 2.f * (s[0] * s[0] + s[1] * s[1] + s[2] * s[2]) + (A[0] + A[4] + A[8]) + (B[0] + B[4] + B[8]);
  float G[9];
  for (int k = 0; k < 9; ++k) G[k] = (k % 4 == 0) ? 2.f : 0.f;
  for (int w = 0; w < 2; ++w) {
    float C[9], V[9];
    sandwich(Hh, w == 0 ? A : B, C);
    jacobi3(C, V);
    const float r[3] = {sqrtf(fmaxf(C[0], 0.f)), sqrtf(fmaxf(C[4], 0.f)), sqrtf(fmaxf(C[8], 0.f))};
    f -= 2.f * (r[0] + r[1] + r[2]);
    float Ch[9], T[9];
    rdrt9(V, r, Ch);
    sandwich(Hi, Ch, T);
    for (int k = 0; k < 9; ++k) G[k] -= T[k];
  }
  if (gsig) {
    float n2 = 0.f;
    for (int k = 0; k < 9; ++k) n2 += G[k] * G[k];
    *gsig = sqrtf(n2);
  }
  // dSk = G  ->  s: 2 s_k (R^T G R)_kk ;  R: 2 G R diag(s^2)  ->  q (through the normalisation)
  float GR[9];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) GR[3 * a + b] = G[3 * a] * R[b] + G[3 * a + 1] * R[3 + b] + G[3 * a + 2] * R[6 + b];
  float dR[9];
  for (int k = 0; k < 3; ++k) {
    g[4 + k] = 2.f * s[k] * (R[k] * GR[k] + R[3 + k] * GR[3 + k] + R[6 + k] * GR[6 + k]);
    for (int a = 0; a < 3; ++a) dR[3 * a + k] = 2.f * GR[3 * a + k] * s[k] * s[k];
  }
  float dq[4];
  quat_rot_vjp(qn, dR, dq);
  const float dot = dq[0] * qn[0] + dq[1] * qn[1] + dq[2] * qn[2] + dq[3] * qn[3];
  for (int k = 0; k < 4; ++k) g[k] = (dq[k] - qn[k] * dot) * iq;
  return f;
}

// Minimise from th (Eq. 10 start); returns the iterations taken.  Stops when the
// gradient has dropped by 1e6 or after kLbfgsIters iterations.  The objective is convex
// in Sk, but the (q, s) parametrisation loses rank where two scales are equal (a
// rotation mixing those axes leaves Sk unchanged), so the (q, s) gradient can vanish
// away from the minimum; when it does while the gradient in Sk has not dropped by 1e3,
// the scales are offset again by the Eq. 10 deltas and the memory is cleared (at most
// three times).  The line search looks
// only at the directional derivative g(x + a d).d (bisection until it is within half of
// the initial slope): near the minimum the objective is a difference of terms ~1e3
// times larger, so float32 values of f can no longer rank two nearby points while the
// gradient still can.
__device__ int lbfgs_w2(float th[7], const float A[9], const float B[9]) {
  float S[kLbfgsMem][7], Y[kLbfgsMem][7], rho[kLbfgsMem];
  int nm = 0, head = 0, it = 0;
  float g[7], gn[7], xn[7], dir[7], gsig0 = 0.f, gsig = 0.f;
  w2_objective(th, A, B, g, &gsig0);
  float g0 = 0.f;
  for (int c = 0; c < 7; ++c) g0 += g[c] * g[c];
  g0 = sqrtf(g0);
  int restarts = 0;
  for (; it < kLbfgsIters; ++it) {
    float gnorm = 0.f;
    for (int c = 0; c < 7; ++c) gnorm += g[c] * g[c];
    gnorm = sqrtf(gnorm);
    if (!(gnorm > 1e-6f * g0) || gnorm == 0.f) {
      w2_objective(th, A, B, g, &gsig);
      if (!(gsig > 1e-3f * gsig0) || restarts == 3) break;
      ++restarts;  // a rank-deficient point of (q, s), not the minimum
      const float delta[3] = {0.001f, 0.002f, 0.003f};
      for (int k = 0; k < 3; ++k) th[4 + k] += delta[k];
      nm = 0;
      w2_objective(th, A, B, g);
      continue;
    }
    // two-loop recursion over the stored pairs, newest first
    float q[7], al[kLbfgsMem];
    for (int c = 0; c < 7; ++c) q[c] = g[c];
    for (int k = 0; k < nm; ++k) {
      const int m = (head - 1 - k + kLbfgsMem) % kLbfgsMem;
      float d = 0.f;
      for (int c = 0; c < 7; ++c) d += S[m][c] * q[c];
      al[m] = rho[m] * d;
      for (int c = 0; c < 7; ++c) q[c] -= al[m] * Y[m][c];
    }
    float gamma;
    if (nm > 0) {
      const int m = (head - 1 + kLbfgsMem) % kLbfgsMem;
      float sy = 0.f, yy = 0.f;
      for (int c = 0; c < 7; ++c) { sy += S[m][c] * Y[m][c]; yy += Y[m][c] * Y[m][c]; }
      gamma = sy / yy;
    } else {
      gamma = 1e-3f / gnorm;
    }
    for (int c = 0; c < 7; ++c) q[c] *= gamma;
    for (int k = nm - 1; k >= 0; --k) {
      const int m = (head - 1 - k + kLbfgsMem) % kLbfgsMem;
      float d = 0.f;
      for (int c = 0; c < 7; ++c) d += Y[m][c] * q[c];
      const float beta = rho[m] * d;
      for (int c = 0; c < 7; ++c) q[c] += S[m][c] * (al[m] - beta);
    }
    float slope = 0.f;
    for (int c = 0; c < 7; ++c) { dir[c] = -q[c]; slope += dir[c] * g[c]; }
    if (!(slope < 0.f)) {  // not a descent direction: drop the memory, steepest descent
      nm = 0;
      slope = 0.f;
      for (int c = 0; c < 7; ++c) { dir[c] = -g[c] * (1e-3f / gnorm); slope += dir[c] * g[c]; }
    }
    // largest step that keeps every scale above a tenth of its magnitude: Sk is singular
    // at s_k = 0, and an iterate that crosses it does not come back
    float amax = 1024.f;
    for (int k = 0; k < 3; ++k) {
      const float sk = th[4 + k], dk = dir[4 + k];
      if (sk * dk < 0.f) amax = fminf(amax, 0.9f * fabsf(sk) / fabsf(dk));
    }
    float step = fminf(1.f, amax), lo = 0.f, hi = -1.f;
    bool ok = false;
    for (int ls = 0; ls < 40; ++ls) {
      for (int c = 0; c < 7; ++c) xn[c] = th[c] + step * dir[c];
      w2_objective(xn, A, B, gn);
      float dd = 0.f;
      for (int c = 0; c < 7; ++c) dd += gn[c] * dir[c];
      if (fabsf(dd) <= 0.5f * fabsf(slope)) { ok = true; break; }
      if (dd < 0.f) {  // still descending: move out, up to amax
        lo = step;
        step = hi < 0.f ? fminf(2.f * step, amax) : 0.5f * (lo + hi);
        if (step == lo) { ok = true; break; }
      } else {  // past the minimum along dir, or not finite: move in
        hi = step;
        step = 0.5f * (lo + hi);
      }
    }
    if (!ok) {
      if (lo == 0.f) break;  // no step along dir lowers the slope: stalled
      for (int c = 0; c < 7; ++c) xn[c] = th[c] + lo * dir[c];  // last point that still descended
      w2_objective(xn, A, B, gn);
    }
    float sv[7], yv[7], sy = 0.f;
    for (int c = 0; c < 7; ++c) {
      sv[c] = xn[c] - th[c];
      yv[c] = gn[c] - g[c];
      sy += sv[c] * yv[c];
    }
    if (sy > 0.f) {  // store the pair (over the oldest one when the memory is full)
      for (int c = 0; c < 7; ++c) { S[head][c] = sv[c]; Y[head][c] = yv[c]; }
      rho[head] = 1.f / sy;
      head = (head + 1) % kLbfgsMem;
      nm = min(nm + 1, kLbfgsMem);
    }
    for (int c = 0; c < 7; ++c) { th[c] = xn[c]; g[c] = gn[c]; }
  }
  return it;
}

// Merge of G_i (older) and G_j: Eq. 6 mean and the closed-form minimiser of Eq. 9,
// computed in the eigenbasis of Sigma_i where Sigma_i = diag(si^2).  solver = 1 takes
// the minimiser of Eq. 9 from the paper's L-BFGS instead (same frame, Eq. 10 start).
// *iters (optional) receives the L-BFGS iterations.
template <int SOLVER>
__device__ void merge_pair(const float* means, const Geom& geo, int64_t i, int64_t j,
                           float mk[3], float qk[4], float lk[3], int* iters = nullptr) {
  float qi[4], si[3], qj[4], sj[3], Ri[9], Rj[9];
  load_qs(geo, i, qi, si);
  load_qs(geo, j, qj, sj);
  quat_rot(qi, Ri);
  quat_rot(qj, Rj);
  // Sigma_j in the basis of R_i: Bj = Ri^T Rj diag(sj^2) Rj^T Ri
  float Mr[9];  // Ri^T Rj
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) Mr[3 * a + b] = Ri[a] * Rj[b] + Ri[3 + a] * Rj[3 + b] + Ri[6 + a] * Rj[6 + b];
  float sj2[3] = {sj[0] * sj[0], sj[1] * sj[1], sj[2] * sj[2]};
  float Bj[9];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      Bj[3 * a + b] = Mr[3 * a] * Mr[3 * b] * sj2[0] + Mr[3 * a + 1] * Mr[3 * b + 1] * sj2[1] + Mr[3 * a + 2] * Mr[3 * b + 2] * sj2[2];
  // Eq. 6 as mu_i + (Pi + Pj)^-1 Pj (mu_j - mu_i), in the R_i basis: Pi = diag(1/si^2).
  float dm[3], dmr[3];
  for (int k = 0; k < 3; ++k) dm[k] = means[3 * j + k] - means[3 * i + k];
  for (int a = 0; a < 3; ++a) dmr[a] = Ri[a] * dm[0] + Ri[3 + a] * dm[1] + Ri[6 + a] * dm[2];
  float Pj[9], isj2[3] = {1.f / sj2[0], 1.f / sj2[1], 1.f / sj2[2]};
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      Pj[3 * a + b] = Mr[3 * a] * Mr[3 * b] * isj2[0] + Mr[3 * a + 1] * Mr[3 * b + 1] * isj2[1] + Mr[3 * a + 2] * Mr[3 * b + 2] * isj2[2];
  float Ps[9];
  for (int k = 0; k < 9; ++k) Ps[k] = Pj[k];
  for (int k = 0; k < 3; ++k) Ps[4 * k] += 1.f / (si[k] * si[k]);
  float rhs[3];
  for (int a = 0; a < 3; ++a) rhs[a] = Pj[3 * a] * dmr[0] + Pj[3 * a + 1] * dmr[1] + Pj[3 * a + 2] * dmr[2];
  float c00 = Ps[4] * Ps[8] - Ps[5] * Ps[7], c01 = Ps[2] * Ps[7] - Ps[1] * Ps[8], c02 = Ps[1] * Ps[5] - Ps[2] * Ps[4];
  float c11 = Ps[0] * Ps[8] - Ps[2] * Ps[6], c12 = Ps[2] * Ps[3] - Ps[0] * Ps[5], c22 = Ps[0] * Ps[4] - Ps[1] * Ps[3];
  float det = Ps[0] * c00 + Ps[1] * (Ps[5] * Ps[6] - Ps[3] * Ps[8]) + Ps[2] * (Ps[3] * Ps[7] - Ps[4] * Ps[6]);
  float id = 1.f / det;
  float xr[3] = {(c00 * rhs[0] + c01 * rhs[1] + c02 * rhs[2]) * id,
                 (c01 * rhs[0] + c11 * rhs[1] + c12 * rhs[2]) * id,
                 (c02 * rhs[0] + c12 * rhs[1] + c22 * rhs[2]) * id};
  for (int k = 0; k < 3; ++k)
    mk[k] = means[3 * i + k] + (Ri[3 * k] * xr[0] + Ri[3 * k + 1] * xr[1] + Ri[3 * k + 2] * xr[2]);
  float Sk[9];  // merged covariance in the R_i basis
  float V[9];
  if constexpr (SOLVER == 1) {
    // Eq. 10 start in this frame: q_i is the identity, q_j the quaternion of R_i^T R_j
    float qr[4];
    rot_quat(Mr, qr);
    const float t = 0.5f;
    const float dq = qr[0];  // <(1,0,0,0), qr>, >= 0: already the shorter arc
    float th[7];
    if (dq > 1.f - 1e-6f) {
      for (int k = 0; k < 4; ++k) th[k] = (1.f - t) * (k == 0 ? 1.f : 0.f) + t * qr[k];
    } else {
      const float om = acosf(fminf(1.f, dq)), so = sinf(om);
      const float ca = sinf((1.f - t) * om) / so, cb = sinf(t * om) / so;
      for (int k = 0; k < 4; ++k) th[k] = ca * (k == 0 ? 1.f : 0.f) + cb * qr[k];
    }
    const float delta[3] = {0.001f, 0.002f, 0.003f};
    for (int k = 0; k < 3; ++k) th[4 + k] = 0.5f * (si[k] + sj[k]) + delta[k];
    float Ai[9] = {si[0] * si[0], 0.f, 0.f, 0.f, si[1] * si[1], 0.f, 0.f, 0.f, si[2] * si[2]};
    const int n_it = lbfgs_w2(th, Ai, Bj);
    if (iters) *iters = n_it;
    const float iq = rsqrtf(th[0] * th[0] + th[1] * th[1] + th[2] * th[2] + th[3] * th[3]);
    const float qn[4] = {th[0] * iq, th[1] * iq, th[2] * iq, th[3] * iq};
    float Rk[9];
    quat_rot(qn, Rk);
    const float s2[3] = {th[4] * th[4], th[5] * th[5], th[6] * th[6]};
    rdrt9(Rk, s2, Sk);
  } else {
  // X = (D Bj D)^(1/2), D = diag(si); Tm = D^-1 X D^-1; Mk = (I + Tm)/2; Sk = Mk D^2 Mk.
  float A[9];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) A[3 * a + b] = si[a] * Bj[3 * a + b] * si[b];
  jacobi3(A, V);
  float ev[3] = {sqrtf(fmaxf(A[0], 0.f)), sqrtf(fmaxf(A[4], 0.f)), sqrtf(fmaxf(A[8], 0.f))};
  float Mk[9];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      float x = V[3 * a] * V[3 * b] * ev[0] + V[3 * a + 1] * V[3 * b + 1] * ev[1] + V[3 * a + 2] * V[3 * b + 2] * ev[2];
      Mk[3 * a + b] = 0.5f * ((a == b ? 1.f : 0.f) + x / (si[a] * si[b]));
    }
  for (int a = 0; a < 3; ++a)  // Mk diag(si^2) Mk, still in the R_i basis
    for (int b = a; b < 3; ++b) {
      float x = 0.f;
      for (int k = 0; k < 3; ++k) x += Mk[3 * a + k] * si[k] * si[k] * Mk[3 * k + b];
      Sk[3 * a + b] = Sk[3 * b + a] = x;
    }
  }
  // eigen-decomposition of Sk -> (quaternion, scales), scales descending, det +1
  jacobi3(Sk, V);
  float lam[3] = {Sk[0], Sk[4], Sk[8]};
  int o0 = 0, o1 = 1, o2 = 2;
  if (lam[o0] < lam[o1]) { int tmp = o0; o0 = o1; o1 = tmp; }
  if (lam[o1] < lam[o2]) { int tmp = o1; o1 = o2; o2 = tmp; }
  if (lam[o0] < lam[o1]) { int tmp = o0; o0 = o1; o1 = tmp; }
  int ord[3] = {o0, o1, o2};
  float E[9];  // world-frame eigenvectors in columns: Ri * V[:, ord]
  for (int c = 0; c < 3; ++c)
    for (int r = 0; r < 3; ++r)
      E[3 * r + c] = Ri[3 * r] * V[ord[c]] + Ri[3 * r + 1] * V[3 + ord[c]] + Ri[3 * r + 2] * V[6 + ord[c]];
  float dE = E[0] * (E[4] * E[8] - E[5] * E[7]) - E[1] * (E[3] * E[8] - E[5] * E[6]) + E[2] * (E[3] * E[7] - E[4] * E[6]);
  if (dE < 0.f)
    for (int r = 0; r < 3; ++r) E[3 * r + 2] = -E[3 * r + 2];
  rot_quat(E, qk);
  for (int c = 0; c < 3; ++c) lk[c] = 0.5f * logf(fmaxf(lam[ord[c]], 1e-30f));
}

template <typename T>
__global__ void __launch_bounds__(256) k_voxel_prep(int64_t n, const float* __restrict__ means, float voxel,
                                                    mgs_merge_params p, int32_t* __restrict__ vox, int32_t* hdr) {
  // Grid-stride over the Gaussians; the bounding box, the eligible count and the
  // overflow flag are reduced per block and folded into hdr with one set of atomics.
  int mn[3] = {INT32_MAX, INT32_MAX, INT32_MAX}, mx[3] = {INT32_MIN, INT32_MIN, INT32_MIN};
  int elig = 0, bad = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    bool e = true;
    if (p.grad_stat) {
      float gs = p.grad_stat[i];
      if (p.vis_count) gs = p.vis_count[i] > 0.f ? __fdiv_rn(gs, p.vis_count[i]) : 0.f;  // Eq. 3 mean
      e = e && gs < p.grad_tau;
    }
    if (p.kf_id) e = e && p.kf_id[i] >= p.kf_min && p.kf_id[i] <= p.kf_max;
    if (e) {
      for (int k = 0; k < 3; ++k) {
        float q = floorf(__fdiv_rn(means[3 * i + k], voxel));
        if (!(q >= -1048576.f && q < 1048576.f)) { bad = 1; q = 0.f; }
        int c = (int)q;
        vox[3 * i + k] = c;
        mn[k] = min(mn[k], c);
        mx[k] = max(mx[k], c);
      }
      ++elig;
    } else {
      for (int k = 0; k < 3; ++k) vox[3 * i + k] = INT32_MIN;
    }
  }
  for (int o = 16; o; o >>= 1) {
    for (int k = 0; k < 3; ++k) {
      mn[k] = min(mn[k], __shfl_xor_sync(0xffffffffu, mn[k], o));
      mx[k] = max(mx[k], __shfl_xor_sync(0xffffffffu, mx[k], o));
    }
    elig += __shfl_xor_sync(0xffffffffu, elig, o);
    bad |= __shfl_xor_sync(0xffffffffu, bad, o);
  }
  __shared__ int s_red[8][8];
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    for (int k = 0; k < 3; ++k) { s_red[w][k] = mn[k]; s_red[w][3 + k] = mx[k]; }
    s_red[w][6] = elig;
    s_red[w][7] = bad;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    for (int ww = 1; ww < nw; ++ww) {
      for (int k = 0; k < 3; ++k) {
        s_red[0][k] = min(s_red[0][k], s_red[ww][k]);
        s_red[0][3 + k] = max(s_red[0][3 + k], s_red[ww][3 + k]);
      }
      s_red[0][6] += s_red[ww][6];
      s_red[0][7] |= s_red[ww][7];
    }
    if (s_red[0][6]) {
      for (int k = 0; k < 3; ++k) {
        atomicMin(&hdr[k], s_red[0][k]);
        atomicMax(&hdr[3 + k], s_red[0][3 + k]);
      }
      atomicAdd(&hdr[6], s_red[0][6]);
      if (s_red[0][7]) atomicOr(&hdr[7], 1);
    }
  }
}

// The key layout from the bounding box of the occupied voxels, on the device (no host
// round trip): bits per axis in hdr[15] = by << 8 | bz.  A box that needs more than 31
// key bits, or a coordinate outside +-2^20 (flag 1 of hdr[7]), sets flag 4: then no
// Gaussian is eligible (hdr[6] = 0) and nothing merges.
__global__ void k_merge_plan(int32_t* hdr) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  auto bits_of = [](int64_t range) { int b = 0; while (b < 40 && (int64_t(1) << b) < range) ++b; return b; };
  const int64_t n_elig = hdr[6];
  int bx = 0, by = 0, bz = 0;
  if (n_elig > 0) {
    bx = bits_of((int64_t)hdr[3] - hdr[0] + 1);
    by = bits_of((int64_t)hdr[4] - hdr[1] + 1);
    bz = bits_of((int64_t)hdr[5] - hdr[2] + 1);
  }
  if ((hdr[7] & 1) || bx + by + bz > 31) {
    hdr[7] |= 4;
    hdr[6] = 0;
    by = bz = 0;
  }
  hdr[15] = (by << 8) | bz;
}

__global__ void k_voxel_pack(int64_t n, const int32_t* __restrict__ vox, const int32_t* __restrict__ hdr,
                             uint32_t* __restrict__ keys) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int x = vox[3 * i];
  if (x == INT32_MIN || (hdr[7] & 4)) { keys[i] = kNoKey; return; }
  const int by = hdr[15] >> 8, bz = hdr[15] & 0xff;
  uint32_t rx = (uint32_t)(x - hdr[0]), ry = (uint32_t)(vox[3 * i + 1] - hdr[1]), rz = (uint32_t)(vox[3 * i + 2] - hdr[2]);
  keys[i] = (rx << (by + bz)) | (ry << bz) | rz;
}

// Grouping by voxel: members only need to be contiguous per voxel (the pairing ranks
// them by (birth, index) itself), so an open-addressing hash table of packed voxel keys
// replaces a sort.  Each eligible Gaussian finds or claims its key's slot (linear
// probing; the table has at least twice as many slots as Gaussians, so a free slot is
// always reached) and takes a rank in it with one atomic; a scan of the slot counts
// gives each slot's first position, and voxels with two or more members are listed as
// (first, end) segments in any order.
__device__ __forceinline__ uint32_t voxel_hash(uint32_t key) {
  key ^= key >> 16;
  key *= 0x7feb352du;
  key ^= key >> 15;
  key *= 0x846ca68bu;
  return key ^ (key >> 16);
}

__global__ void k_hash_insert(int64_t n, const uint32_t* __restrict__ keys, uint32_t* tkey,
                              uint32_t* __restrict__ tcount, uint32_t tmask, uint32_t* __restrict__ slot,
                              uint32_t* __restrict__ rank, int32_t* __restrict__ hdr) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t key = keys[i];
  if (key == kNoKey) { slot[i] = kNoKey; return; }
  uint32_t h = voxel_hash(key) & tmask;
  for (uint32_t probe = 0; probe <= tmask; ++probe) {
    uint32_t cur = *(volatile uint32_t*)&tkey[h];
    if (cur == kNoKey) cur = atomicCAS(&tkey[h], kNoKey, key);
    if (cur == kNoKey || cur == key) {
      slot[i] = h;
      rank[i] = atomicAdd(&tcount[h], 1u);
      return;
    }
    h = (h + 1) & tmask;
  }
  slot[i] = kNoKey;  // the table is full: cannot happen with >= 2n slots
  atomicOr(&hdr[7], 8);
}

__global__ void k_hash_scatter(int64_t n, const uint32_t* __restrict__ slot, const uint32_t* __restrict__ rank,
                               const uint32_t* __restrict__ toff, uint32_t* __restrict__ perm) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t s = slot[i];
  if (s != kNoKey) perm[toff[s] + rank[i]] = (uint32_t)i;
}

// One atomic on the voxel counter per block (its warps' counts meet in shared memory):
// one per warp serialised tens of thousands of atomics on a single address.
__global__ void __launch_bounds__(256) k_hash_segs(uint32_t tsize, const uint32_t* __restrict__ tcount,
                                                   const uint32_t* __restrict__ toff, uint2* __restrict__ segs,
                                                   uint32_t* __restrict__ n_vox) {
  __shared__ uint32_t s_cnt[8], s_base;
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t c = t < tsize ? tcount[t] : 0u;
  const bool multi = c >= 2;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint32_t mask = __ballot_sync(0xffffffffu, multi);
  if (lane == 0) s_cnt[w] = (uint32_t)__popc(mask);
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t tot = 0;
    for (int k = 0; k < 8; ++k) {
      const uint32_t x = s_cnt[k];
      s_cnt[k] = tot;
      tot += x;
    }
    s_base = tot ? atomicAdd(n_vox, tot) : 0u;
  }
  __syncthreads();
  if (multi) {
    const uint32_t f = toff[t];
    segs[s_base + s_cnt[w] + __popc(mask & ((1u << lane) - 1u))] = make_uint2(f, f + c);
  }
}

struct PairCand {
  float d2;
  int a, b;  // member ranks (a older)
};

// Pairing of the voxels with 2..32 members (larger ones go to the block path).
// Members are ranked by (birth, index), Eq. 4 is evaluated for every older/younger
// pair, and pairs below chi2 are taken greedily on (d2, birth_i, birth_j, i, j).
// A warp takes four consecutive voxels at a time: voxels with at most 8 members are
// paired by 8-lane groups side by side (all shuffles run on the whole warp with fixed
// trip counts; a group's lanes reduce among themselves), larger ones by the whole warp
// one after the other.
constexpr int kGroupVoxel = 8;

template <typename T>
__global__ void __launch_bounds__(128) k_voxel_pairs(
    const float* __restrict__ means, const Geom geo,
    const uint64_t* __restrict__ birth, const uint32_t* __restrict__ perm,
    const uint2* __restrict__ segs, const uint32_t* __restrict__ n_vox_p, float chi2, int greedy,
    int32_t* __restrict__ partner, uint2* __restrict__ pairs, uint32_t* __restrict__ n_pairs,
    uint32_t* __restrict__ big, uint32_t* __restrict__ n_big) {
  __shared__ float s_d2[4][kWarpVoxel][kWarpVoxel + 1];
  __shared__ float s_mu[4][kWarpVoxel][3];   // member means, by rank
  __shared__ float s_P[4][kWarpVoxel][7];    // member precisions (6 used, odd stride), by rank
  __shared__ int64_t s_idx[4][kWarpVoxel];
  __shared__ uint64_t s_birth[4][kWarpVoxel];
  __shared__ int s_pairs[4][kWarpVoxel / 2][2];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t n_vox = (int64_t)*n_vox_p;
  // whole-warp pairing of voxel v (2..32 members; more go to the big list)
  auto warp_voxel = [&](int64_t v) {
  const uint2 sg = segs[v];
  const uint32_t st = sg.x;
  const int nm = (int)(sg.y - sg.x);
  if (nm > kWarpVoxel) {
    if (lane == 0) big[atomicAdd(n_big, 1u)] = (uint32_t)v;
    return;
  }
  // each lane loads its own member (independent loads), then places it by rank
  int64_t my = lane < nm ? (int64_t)perm[st + lane] : -1;
  uint64_t mb = ~0ull;
  float P[6], mu[3];
  if (lane < nm) {
    mb = birth[my];
    precision_of(geo, my, P);
    mu[0] = means[3 * my]; mu[1] = means[3 * my + 1]; mu[2] = means[3 * my + 2];
  }
  int rank = 0;
  for (int m = 0; m < nm; ++m) {
    int64_t oi = __shfl_sync(0xffffffffu, my, m);
    uint64_t ob = __shfl_sync(0xffffffffu, mb, m);
    if (lane < nm && older(ob, oi, mb, my)) ++rank;
  }
  if (lane < nm) {
    s_idx[wib][rank] = my;
    s_birth[wib][rank] = mb;
#pragma unroll
    for (int k = 0; k < 3; ++k) s_mu[wib][rank][k] = mu[k];
#pragma unroll
    for (int k = 0; k < 6; ++k) s_P[wib][rank][k] = P[k];
  }
  __syncwarp();
  // Eq. 4 rows: lane a (older) against every younger b
  if (lane < nm) {
    float Pa[6], mav[3];
#pragma unroll
    for (int k = 0; k < 6; ++k) Pa[k] = s_P[wib][lane][k];
#pragma unroll
    for (int k = 0; k < 3; ++k) mav[k] = s_mu[wib][lane][k];
    for (int b = lane + 1; b < nm; ++b) s_d2[wib][lane][b] = mahalanobis2(Pa, mav, s_mu[wib][b]);
  }
  __syncwarp();
  uint32_t matched = 0;
  int np = 0;
  for (int round = 0; round < nm / 2; ++round) {
    PairCand best{INFINITY, -1, -1};
    if (lane < nm && !((matched >> lane) & 1u)) {
      for (int b = lane + 1; b < nm; ++b) {
        if ((matched >> b) & 1u) continue;
        float d2 = s_d2[wib][lane][b];
        if (d2 < chi2 && d2 < best.d2) best = PairCand{d2, lane, b};  // lane fixed: later b has later rank
      }
    }
    for (int o = 16; o; o >>= 1) {
      PairCand oc{__shfl_xor_sync(0xffffffffu, best.d2, o), __shfl_xor_sync(0xffffffffu, best.a, o),
                  __shfl_xor_sync(0xffffffffu, best.b, o)};
      bool take;
      if (oc.a < 0) take = false;
      else if (best.a < 0) take = true;
      else if (oc.d2 != best.d2) take = oc.d2 < best.d2;
      else {
        uint64_t b1 = s_birth[wib][best.a], b2 = s_birth[wib][best.b];
        uint64_t c1 = s_birth[wib][oc.a], c2 = s_birth[wib][oc.b];
        int64_t i1 = s_idx[wib][best.a], i2 = s_idx[wib][best.b];
        int64_t j1 = s_idx[wib][oc.a], j2 = s_idx[wib][oc.b];
        if (c1 != b1) take = c1 < b1;
        else if (c2 != b2) take = c2 < b2;
        else if (j1 != i1) take = j1 < i1;
        else take = j2 < i2;
      }
      if (take) best = oc;
    }
    if (best.a < 0) break;
    matched |= (1u << best.a) | (1u << best.b);
    if (lane == 0) { s_pairs[wib][np][0] = best.a; s_pairs[wib][np][1] = best.b; }
    ++np;
    if (!greedy) break;
  }
  __syncwarp();
  uint32_t slot = 0;
  if (lane == 0 && np > 0) slot = atomicAdd(n_pairs, (uint32_t)np);
  slot = __shfl_sync(0xffffffffu, slot, 0);
  if (lane < np) {
    int64_t i = s_idx[wib][s_pairs[wib][lane][0]], j = s_idx[wib][s_pairs[wib][lane][1]];
    partner[i] = (int32_t)j;
    partner[j] = (int32_t)i;
    pairs[slot + lane] = make_uint2((uint32_t)i, (uint32_t)j);
  }
  __syncwarp();  // the warp's shared rows are reused by its next voxel
  };
  const int grp = lane >> 3, gl = lane & (kGroupVoxel - 1), gbase = grp * kGroupVoxel;
  // Persistent warps: warp-stride loop over groups of four voxels.
  for (int64_t vg = ((int64_t)blockIdx.x * 4 + wib) * 4; vg < n_vox; vg += (int64_t)gridDim.x * 16) {
    const int64_t v = vg + grp;
    uint32_t st = 0;
    int nm = 0;
    if (v < n_vox) {
      const uint2 sg = segs[v];
      st = sg.x;
      nm = (int)(sg.y - sg.x);
    }
    const bool small = nm >= 2 && nm <= kGroupVoxel;
    const bool mine = small && gl < nm;
    // each lane loads its own member (independent loads), then places it by rank
    const int64_t my = mine ? (int64_t)perm[st + gl] : -1;
    uint64_t mb = ~0ull;
    float P[6], mu[3];
    if (mine) {
      mb = birth[my];
      precision_of(geo, my, P);
      mu[0] = means[3 * my]; mu[1] = means[3 * my + 1]; mu[2] = means[3 * my + 2];
    }
    int rank = 0;
#pragma unroll
    for (int m = 0; m < kGroupVoxel; ++m) {
      const int64_t oi = __shfl_sync(0xffffffffu, my, gbase + m);
      const uint64_t ob = __shfl_sync(0xffffffffu, mb, gbase + m);
      if (mine && m < nm && older(ob, oi, mb, my)) ++rank;
    }
    if (mine) {
      s_idx[wib][gbase + rank] = my;
      s_birth[wib][gbase + rank] = mb;
#pragma unroll
      for (int k = 0; k < 3; ++k) s_mu[wib][gbase + rank][k] = mu[k];
#pragma unroll
      for (int k = 0; k < 6; ++k) s_P[wib][gbase + rank][k] = P[k];
    }
    __syncwarp();
    if (mine) {  // Eq. 4 row: rank gl (older) against every younger rank
      float Pa[6], mav[3];
#pragma unroll
      for (int k = 0; k < 6; ++k) Pa[k] = s_P[wib][gbase + gl][k];
#pragma unroll
      for (int k = 0; k < 3; ++k) mav[k] = s_mu[wib][gbase + gl][k];
      for (int b = gl + 1; b < nm; ++b) s_d2[wib][gbase + gl][b] = mahalanobis2(Pa, mav, s_mu[wib][gbase + b]);
    }
    __syncwarp();
    uint32_t matched = 0;
    int np = 0;
    bool done = !small;
    for (int round = 0; round < kGroupVoxel / 2; ++round) {
      PairCand best{INFINITY, -1, -1};
      if (!done && gl < nm && !((matched >> gl) & 1u)) {
        for (int b = gl + 1; b < nm; ++b) {
          if ((matched >> b) & 1u) continue;
          const float d2 = s_d2[wib][gbase + gl][b];
          if (d2 < chi2 && d2 < best.d2) best = PairCand{d2, gl, b};
        }
      }
      for (int o = kGroupVoxel / 2; o; o >>= 1) {  // stays inside the 8-lane group
        PairCand oc{__shfl_xor_sync(0xffffffffu, best.d2, o), __shfl_xor_sync(0xffffffffu, best.a, o),
                    __shfl_xor_sync(0xffffffffu, best.b, o)};
        bool take;
        if (oc.a < 0) take = false;
        else if (best.a < 0) take = true;
        else if (oc.d2 != best.d2) take = oc.d2 < best.d2;
        else {
          const uint64_t b1 = s_birth[wib][gbase + best.a], b2 = s_birth[wib][gbase + best.b];
          const uint64_t c1 = s_birth[wib][gbase + oc.a], c2 = s_birth[wib][gbase + oc.b];
          const int64_t i1 = s_idx[wib][gbase + best.a], i2 = s_idx[wib][gbase + best.b];
          const int64_t j1 = s_idx[wib][gbase + oc.a], j2 = s_idx[wib][gbase + oc.b];
          if (c1 != b1) take = c1 < b1;
          else if (c2 != b2) take = c2 < b2;
          else if (j1 != i1) take = j1 < i1;
          else take = j2 < i2;
        }
        if (take) best = oc;
      }
      if (!done) {
        if (best.a < 0) {
          done = true;
        } else {
          matched |= (1u << best.a) | (1u << best.b);
          if (gl == 0) {
            s_pairs[wib][grp * (kGroupVoxel / 2) + np][0] = best.a;
            s_pairs[wib][grp * (kGroupVoxel / 2) + np][1] = best.b;
          }
          ++np;
          if (!greedy || np == nm / 2) done = true;
        }
      }
      if (__all_sync(0xffffffffu, done)) break;
    }
    __syncwarp();
    uint32_t slot = 0;
    {  // one atomic per warp for the pairs of its groups (np is uniform within a group)
      uint32_t tot = 0, pre = 0;
#pragma unroll
      for (int q = 0; q < 32 / kGroupVoxel; ++q) {
        const uint32_t x = (uint32_t)__shfl_sync(0xffffffffu, np, q * kGroupVoxel);
        if (q < grp) pre += x;
        tot += x;
      }
      uint32_t base = 0;
      if (lane == 0 && tot) base = atomicAdd(n_pairs, tot);
      slot = __shfl_sync(0xffffffffu, base, 0) + pre;
    }
    if (gl < np) {
      const int64_t i = s_idx[wib][gbase + s_pairs[wib][grp * (kGroupVoxel / 2) + gl][0]];
      const int64_t j = s_idx[wib][gbase + s_pairs[wib][grp * (kGroupVoxel / 2) + gl][1]];
      partner[i] = (int32_t)j;
      partner[j] = (int32_t)i;
      pairs[slot + gl] = make_uint2((uint32_t)i, (uint32_t)j);
    }
    __syncwarp();  // the groups' shared rows are reused below and by the next voxels
    uint32_t large = __ballot_sync(0xffffffffu, gl == 0 && nm > kGroupVoxel);
    while (large) {
      const int src = __ffs(large) - 1;
      large &= large - 1;
      warp_voxel(vg + (src >> 3));
    }
  }
}

// Block path: a voxel with 33..256 members; d2 evaluated on the fly each round.
template <typename T>
__global__ void __launch_bounds__(kBlockVoxel) k_voxel_pairs_big(
    const float* __restrict__ means, const Geom geo,
    const uint64_t* __restrict__ birth, const uint32_t* __restrict__ perm,
    const uint2* __restrict__ segs, const uint32_t* __restrict__ big,
    const uint32_t* __restrict__ n_big_p, float chi2, int greedy, int32_t* __restrict__ partner,
    uint2* __restrict__ pairs, uint32_t* __restrict__ n_pairs, uint32_t* __restrict__ huge,
    uint32_t* __restrict__ n_huge) {
  __shared__ int64_t s_idx[kBlockVoxel];
  __shared__ uint64_t s_birth[kBlockVoxel];
  __shared__ float s_mu[kBlockVoxel][3];
  __shared__ float s_P[kBlockVoxel][6];
  __shared__ int s_match[kBlockVoxel];
  __shared__ float r_d2[kBlockVoxel];
  __shared__ int r_a[kBlockVoxel], r_b[kBlockVoxel];
  __shared__ int s_pairs[kBlockVoxel / 2][2];
  __shared__ int s_np;
  __shared__ uint32_t s_slot;
  const uint32_t n_big = *n_big_p;
  const int t = threadIdx.x;
  // Block-stride loop over the big voxels (every branch below is uniform per block).
  for (uint32_t bv = blockIdx.x; bv < n_big; bv += gridDim.x) {
  const uint32_t v = big[bv];
  const uint32_t st = segs[v].x, en = segs[v].y;
  const int nm = (int)(en - st);
  if (nm > kBlockVoxel) {  // left to the global-memory path
    if (t == 0) huge[atomicAdd(n_huge, 1u)] = v;
    continue;
  }
  int64_t my = t < nm ? (int64_t)perm[st + t] : -1;
  uint64_t mb = t < nm ? birth[my] : ~0ull;
  if (t < nm) { s_idx[t] = my; s_birth[t] = mb; }
  __syncthreads();
  int rank = 0;
  if (t < nm)
    for (int m = 0; m < nm; ++m)
      if (older(s_birth[m], s_idx[m], mb, my)) ++rank;
  __syncthreads();
  if (t < nm) {
    s_idx[rank] = my;
    s_birth[rank] = mb;
    s_match[rank] = 0;
    for (int k = 0; k < 3; ++k) s_mu[rank][k] = means[3 * my + k];
    precision_of(geo, my, s_P[rank]);
  }
  if (t == 0) s_np = 0;
  __syncthreads();
  const int npairs = nm * (nm - 1) / 2;
  for (int round = 0; round < nm / 2; ++round) {
    float bd = INFINITY;
    int ba = -1, bb = -1;
    for (int pi = t; pi < npairs; pi += kBlockVoxel) {
      // decode pair index -> (a, b), a < b
      int a = 0, rem = pi;
      while (rem >= nm - 1 - a) { rem -= nm - 1 - a; ++a; }
      int b = a + 1 + rem;
      if (s_match[a] || s_match[b]) continue;
      float d2 = mahalanobis2(s_P[a], s_mu[a], s_mu[b]);
      if (d2 >= chi2) continue;
      bool take = ba < 0 || d2 < bd || (d2 == bd && (a < ba || (a == ba && b < bb)));
      if (take) { bd = d2; ba = a; bb = b; }
    }
    r_d2[t] = bd; r_a[t] = ba; r_b[t] = bb;
    __syncthreads();
    for (int stp = kBlockVoxel / 2; stp; stp >>= 1) {
      if (t < stp) {
        int oa = r_a[t + stp];
        bool take;
        if (oa < 0) take = false;
        else if (r_a[t] < 0) take = true;
        else if (r_d2[t + stp] != r_d2[t]) take = r_d2[t + stp] < r_d2[t];
        else take = oa < r_a[t] || (oa == r_a[t] && r_b[t + stp] < r_b[t]);  // rank order = (birth, index)
        if (take) { r_d2[t] = r_d2[t + stp]; r_a[t] = oa; r_b[t] = r_b[t + stp]; }
      }
      __syncthreads();
    }
    int a = r_a[0], b = r_b[0];
    __syncthreads();
    if (a < 0) break;
    if (t == 0) { s_match[a] = 1; s_match[b] = 1; s_pairs[s_np][0] = a; s_pairs[s_np][1] = b; s_np++; }
    __syncthreads();
    if (!greedy) break;
  }
  if (t == 0) s_slot = s_np ? atomicAdd(n_pairs, (uint32_t)s_np) : 0u;
  __syncthreads();
  for (int k = t; k < s_np; k += kBlockVoxel) {
    int64_t i = s_idx[s_pairs[k][0]], j = s_idx[s_pairs[k][1]];
    partner[i] = (int32_t)j;
    partner[j] = (int32_t)i;
    pairs[s_slot + k] = make_uint2((uint32_t)i, (uint32_t)j);
  }
  __syncthreads();  // shared state is reused by the next voxel
  }
}

// Global-memory path: a voxel with more than 256 members, one block per voxel.  The
// members are ranked by (birth, index) into global scratch at the voxel's positions of
// the sorted order; each greedy round takes the block-wide minimum of (d2, rank a,
// rank b) over the unmatched pairs below chi2, as the shared-memory path does.
template <typename T>
__global__ void __launch_bounds__(kBlockVoxel) k_voxel_pairs_huge(
    const float* __restrict__ means, const Geom geo, const uint64_t* __restrict__ birth,
    const uint32_t* __restrict__ perm, const uint2* __restrict__ segs, const uint32_t* __restrict__ huge,
    const uint32_t* __restrict__ n_huge_p, float chi2, int greedy, int32_t* __restrict__ partner,
    uint2* __restrict__ pairs, uint32_t* __restrict__ n_pairs, int64_t* __restrict__ h_idx,
    float* __restrict__ h_mu, float* __restrict__ h_P, int32_t* __restrict__ h_match) {
  __shared__ float r_d2[kBlockVoxel];
  __shared__ int r_a[kBlockVoxel], r_b[kBlockVoxel];
  const uint32_t n_huge = *n_huge_p;
  const int t = threadIdx.x;
  for (uint32_t hv = blockIdx.x; hv < n_huge; hv += gridDim.x) {
    const uint32_t v = huge[hv];
    const uint32_t st = segs[v].x;
    const int nm = (int)(segs[v].y - st);
    for (int m = t; m < nm; m += kBlockVoxel) {
      const int64_t i = perm[st + m];
      const uint64_t bi = birth[i];
      int rank = 0;
      for (int k = 0; k < nm; ++k) {
        const int64_t j = perm[st + k];
        if (older(birth[j], j, bi, i)) ++rank;
      }
      const uint32_t slot = st + (uint32_t)rank;
      h_idx[slot] = i;
      h_match[slot] = 0;
      for (int k = 0; k < 3; ++k) h_mu[3 * (size_t)slot + k] = means[3 * i + k];
      precision_of(geo, i, h_P + 6 * (size_t)slot);
    }
    __syncthreads();
    for (int round = 0; round < nm / 2; ++round) {
      float bd = INFINITY;
      int ba = -1, bb = -1;
      for (int a = t; a < nm; a += kBlockVoxel) {
        if (h_match[st + a]) continue;
        float P[6], ma[3];
        for (int k = 0; k < 6; ++k) P[k] = h_P[6 * (size_t)(st + a) + k];
        for (int k = 0; k < 3; ++k) ma[k] = h_mu[3 * (size_t)(st + a) + k];
        for (int b = a + 1; b < nm; ++b) {
          if (h_match[st + b]) continue;
          const float d2 = mahalanobis2(P, ma, h_mu + 3 * (size_t)(st + b));
          if (d2 >= chi2) continue;
          // a rises with the thread's rows, b within a row: (d2, a, b) order per thread
          if (ba < 0 || d2 < bd || (d2 == bd && (a < ba || (a == ba && b < bb)))) { bd = d2; ba = a; bb = b; }
        }
      }
      r_d2[t] = bd; r_a[t] = ba; r_b[t] = bb;
      __syncthreads();
      for (int stp = kBlockVoxel / 2; stp; stp >>= 1) {
        if (t < stp) {
          const int oa = r_a[t + stp];
          bool take;
          if (oa < 0) take = false;
          else if (r_a[t] < 0) take = true;
          else if (r_d2[t + stp] != r_d2[t]) take = r_d2[t + stp] < r_d2[t];
          else take = oa < r_a[t] || (oa == r_a[t] && r_b[t + stp] < r_b[t]);
          if (take) { r_d2[t] = r_d2[t + stp]; r_a[t] = oa; r_b[t] = r_b[t + stp]; }
        }
        __syncthreads();
      }
      const int a = r_a[0], b = r_b[0];
      __syncthreads();
      if (a < 0) break;
      if (t == 0) {
        h_match[st + a] = 1;
        h_match[st + b] = 1;
        const int64_t i = h_idx[st + a], j = h_idx[st + b];
        partner[i] = (int32_t)j;
        partner[j] = (int32_t)i;
        pairs[atomicAdd(n_pairs, 1u)] = make_uint2((uint32_t)i, (uint32_t)j);
      }
      __syncthreads();
      if (!greedy) break;
    }
    __syncthreads();  // the next voxel's ranking must not overlap this one's last reads
  }
}

// One thread per accepted pair: Eq. 6 mean and the Eq. 9 barycentre, written in the
// older Gaussian's slot of the merged-value arrays.
template <typename T, int SOLVER>
__global__ void __launch_bounds__(128) k_merge_pairs(const float* __restrict__ means, const Geom geo,
                                                     const uint2* __restrict__ pairs,
                                                     const uint32_t* __restrict__ n_pairs_p,
                                                     float* __restrict__ mmean, float* __restrict__ mquat,
                                                     float* __restrict__ mlogs,
                                                     unsigned long long* __restrict__ iters) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= (int64_t)*n_pairs_p) return;
  const uint2 pr = pairs[k];
  const int64_t i = pr.x, j = pr.y;
  float mk[3], qk[4], lk[3];
  int it = 0;
  merge_pair<SOLVER>(means, geo, i, j, mk, qk, lk, &it);
  if (SOLVER == 1 && iters) atomicAdd(iters, (unsigned long long)it);
  for (int c = 0; c < 3; ++c) { mmean[3 * i + c] = mk[c]; mlogs[3 * i + c] = lk[c]; }
  for (int c = 0; c < 4; ++c) mquat[4 * i + c] = qk[c];
}

__global__ void k_keep(int64_t n, const int32_t* __restrict__ partner, const uint64_t* __restrict__ birth,
                       uint32_t* __restrict__ keep) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int32_t j = partner[i];
  keep[i] = (j >= 0 && older(birth[j], j, birth[i], i)) ? 0u : 1u;
}

template <typename T>
__global__ void k_compact(int64_t n, int K3, const float* __restrict__ means, const Geom geo,
                          const T* __restrict__ ol, const T* __restrict__ sh,
                          const uint64_t* __restrict__ birth, const uint32_t* __restrict__ keep,
                          const uint32_t* __restrict__ pos, const int32_t* __restrict__ partner,
                          const float* __restrict__ mmean, const float* __restrict__ mquat,
                          const float* __restrict__ mlogs, float* omeans, void* ols, void* oqs, T* ool,
                          T* osh, uint64_t* obirth) {
  // SH rows: the block copies the rows of its kept Gaussians cooperatively, in 16-byte
  // chunks when both arrays allow it (rows of whole chunks, 16-byte aligned), else
  // element by element; either way consecutive threads touch consecutive addresses.
  {
    const int64_t g0 = (int64_t)blockIdx.x * blockDim.x;
    const int rows = (int)(n - g0 < (int64_t)blockDim.x ? n - g0 : (int64_t)blockDim.x);
    const int row_bytes = K3 * (int)sizeof(T);
    if (row_bytes % 16 == 0 && ((uintptr_t)sh & 15u) == 0 && ((uintptr_t)osh & 15u) == 0) {
      const int Q = row_bytes / 16;
      const uint4* src = reinterpret_cast<const uint4*>(sh);
      uint4* dst = reinterpret_cast<uint4*>(osh);
      for (int c = threadIdx.x; c < rows * Q; c += blockDim.x) {
        const int r = c / Q, q = c - r * Q;
        const int64_t gi = g0 + r;
        if (keep[gi]) dst[(int64_t)pos[gi] * Q + q] = __ldcs(src + gi * Q + q);
      }
    } else {
      for (int c = threadIdx.x; c < rows * K3; c += blockDim.x) {
        const int r = c / K3, k = c - r * K3;
        const int64_t gi = g0 + r;
        if (keep[gi]) osh[(int64_t)pos[gi] * K3 + k] = sh[gi * K3 + k];
      }
    }
  }
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || !keep[i]) return;
  int64_t w = pos[i];
  if (partner[i] >= 0) {
    for (int k = 0; k < 3; ++k) { omeans[3 * w + k] = mmean[3 * i + k]; st_dt(ols, geo.dt, 3 * w + k, mlogs[3 * i + k]); }
    for (int k = 0; k < 4; ++k) st_dt(oqs, geo.qdt, 4 * w + k, mquat[4 * i + k]);
  } else {
    for (int k = 0; k < 3; ++k) { omeans[3 * w + k] = means[3 * i + k]; cp_dt(ols, geo.ls, geo.dt, 3 * w + k, 3 * i + k); }
    for (int k = 0; k < 4; ++k) cp_dt(oqs, geo.qs, geo.qdt, 4 * w + k, 4 * i + k);
  }
  ool[w] = ol[i];
  if (obirth) obirth[w] = birth[i];
}

// The whole merge, asynchronous on s: every launch is sized from n and reads the
// counts it needs (eligible Gaussians, voxels, pairs) from hdr on the device.  The
// survivor count lands in hdr[10], the error flags in hdr[7].
template <typename T>
cudaError_t merge_t(const mgs_gaussians& in, float voxel, const mgs_merge_params& p,
                    const mgs_gaussians_mut& out, int32_t* partner_out, int32_t* vox_out, MergeWs& ws,
                    cudaStream_t s) {
  const int64_t n = in.n;
  const Geom geo{in.log_scales, in.quats, in.geom_dtype, in.quat_dtype};
  const T* ol = (const T*)in.opacity_logit;
  const T* sh = (const T*)in.sh;
  const int K3 = (in.sh_degree + 1) * (in.sh_degree + 1) * 3;
  const unsigned grid = (unsigned)div_up(n, 256);
  static const int32_t init[16] = {INT32_MAX, INT32_MAX, INT32_MAX, INT32_MIN, INT32_MIN, INT32_MIN,
                                   0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  cudaError_t e = cudaMemcpyAsync(ws.hdr, init, sizeof(init), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  int32_t* partner = partner_out ? partner_out : ws.partner;
  e = cudaMemsetAsync(partner, 0xff, sizeof(int32_t) * n, s);
  if (e != cudaSuccess) return e;
  int32_t* vox = vox_out ? vox_out : ws.vox;
  k_voxel_prep<T><<<(unsigned)std::min<int64_t>(grid, kPersistBlocks), 256, 0, s>>>(n, in.means, voxel, p, vox, ws.hdr);
  k_merge_plan<<<1, 32, 0, s>>>(ws.hdr);
  k_voxel_pack<<<grid, 256, 0, s>>>(n, vox, ws.hdr, ws.keys[0]);
  count_launch(3);
  // group the eligible Gaussians by voxel (ineligible ones carry the all-ones key)
  uint32_t* slot = ws.keys[1];
  uint32_t* rank = ws.flags;
  uint32_t* perm_w = ws.perm[0];
  e = cudaMemsetAsync(ws.tkey, 0xff, 4 * (size_t)ws.tsize, s);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(ws.tcount, 0, 4 * (size_t)ws.tsize, s);
  if (e != cudaSuccess) return e;
  k_hash_insert<<<grid, 256, 0, s>>>(n, ws.keys[0], ws.tkey, ws.tcount, ws.tsize - 1, slot, rank, ws.hdr);
  count_launch();
  e = scan_exclusive_u32(ws.tcount, nullptr, ws.toff, (int64_t)ws.tsize, ws.tscratch, nullptr, s);
  if (e != cudaSuccess) return e;
  k_hash_scatter<<<grid, 256, 0, s>>>(n, slot, rank, ws.toff, perm_w);
  uint32_t* n_vox = (uint32_t*)(ws.hdr + 8);
  uint32_t* n_big = (uint32_t*)(ws.hdr + 9);
  k_hash_segs<<<(unsigned)div_up(ws.tsize, 256), 256, 0, s>>>(ws.tsize, ws.tcount, ws.toff, ws.segs, n_vox);
  count_launch(4);  // with the two pairing kernels below
  const uint32_t* perm = perm_w;
  // 8 blocks of 128 threads per SM fit by registers (64) and shared memory (24 KB)
  const unsigned gv = (unsigned)std::min<int64_t>(std::max<int64_t>(1, div_up(n, 4)), kPersistBlocks);
  uint32_t* n_pairs = (uint32_t*)(ws.hdr + 11);
  k_voxel_pairs<T><<<gv, 128, 0, s>>>(in.means, geo, in.birth, perm, ws.segs, n_vox, p.chi2,
                                      p.greedy, partner, ws.pairs, n_pairs, ws.big, n_big);
  uint32_t* n_huge = (uint32_t*)(ws.hdr + 14);
  k_voxel_pairs_big<T><<<(unsigned)std::min<int64_t>(std::max<int64_t>(1, n / 33), 152 * 2), kBlockVoxel, 0, s>>>(
      in.means, geo, in.birth, perm, ws.segs, ws.big, n_big, p.chi2, p.greedy, partner,
      ws.pairs, n_pairs, ws.huge, n_huge);
  k_voxel_pairs_huge<T><<<(unsigned)std::min<int64_t>(std::max<int64_t>(1, n / 257), 152), kBlockVoxel, 0, s>>>(
      in.means, geo, in.birth, perm, ws.segs, ws.huge, n_huge, p.chi2, p.greedy, partner, ws.pairs, n_pairs,
      ws.h_idx, ws.h_mu, ws.h_P, ws.h_match);
  count_launch();
  const unsigned gp = (unsigned)div_up(n / 2 + 1, 128);
  unsigned long long* iters = reinterpret_cast<unsigned long long*>(ws.hdr + 12);
  if (p.solver == 1)
    k_merge_pairs<T, 1><<<gp, 128, 0, s>>>(in.means, geo, ws.pairs, n_pairs, ws.mmean, ws.mquat, ws.mlogs, iters);
  else
    k_merge_pairs<T, 0><<<gp, 128, 0, s>>>(in.means, geo, ws.pairs, n_pairs, ws.mmean, ws.mquat, ws.mlogs, iters);
  count_launch();
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_keep<<<grid, 256, 0, s>>>(n, partner, in.birth, ws.flags);
  count_launch(2);  // with the compaction below
  uint32_t* n_out_dev = (uint32_t*)(ws.hdr + 10);
  e = scan_exclusive_u32(ws.flags, nullptr, ws.pos, n, ws.scratch, n_out_dev, s);
  if (e != cudaSuccess) return e;
  k_compact<T><<<grid, 256, 0, s>>>(n, K3, in.means, geo, ol, sh, in.birth, ws.flags, ws.pos, partner,
                                    ws.mmean, ws.mquat, ws.mlogs, out.means, out.log_scales,
                                    out.quats, (T*)out.opacity_logit, (T*)out.sh, out.birth);
  return cudaGetLastError();
}

}  // namespace

MergeStats& last_merge_stats() {
  static thread_local MergeStats st;
  return st;
}

size_t merge_workspace_bytes(int64_t n, MergeWs* ws, char* base) {
  size_t off = 0;
  auto take = [&](size_t bytes) { char* p = base ? base + off : nullptr; off += align_up(bytes); return p; };
  int64_t m = std::max<int64_t>(n, 1);
  MergeWs w{};
  w.hdr = (int32_t*)take(64);
  w.vox = (int32_t*)take(12 * m);
  w.keys[0] = (uint32_t*)take(4 * m);
  w.keys[1] = (uint32_t*)take(4 * m);
  w.perm[0] = (uint32_t*)take(4 * m);
  w.perm[1] = (uint32_t*)take(4 * m);
  w.flags = (uint32_t*)take(4 * m);
  w.pos = (uint32_t*)take(4 * m);
  w.segs = (uint2*)take(8 * m);
  uint32_t ts = 1024;
  while ((int64_t)ts < 2 * m) ts <<= 1;
  w.tsize = ts;
  w.tkey = (uint32_t*)take(4 * (size_t)ts);
  w.tcount = (uint32_t*)take(4 * (size_t)ts);
  w.toff = (uint32_t*)take(4 * ((size_t)ts + 1));
  w.tscratch = (uint32_t*)take(4 * (size_t)(ts / kSortTile + 4));
  w.partner = (int32_t*)take(4 * m);
  w.mmean = (float*)take(12 * m);
  w.mquat = (float*)take(16 * m);
  w.mlogs = (float*)take(12 * m);
  w.big = (uint32_t*)take(4 * m);
  w.huge = (uint32_t*)take(4 * m);
  w.h_idx = (int64_t*)take(8 * m);
  w.h_mu = (float*)take(12 * m);
  w.h_P = (float*)take(24 * m);
  w.h_match = (int32_t*)take(4 * m);
  w.pairs = (uint2*)take(8 * (m / 2 + 1));
  w.scratch = (uint32_t*)take(4 * sort_scratch_words(m));
  if (ws) *ws = w;
  return off;
}

// Asynchronous merge on s; the survivor count (hdr[10]) and the error flags (hdr[7]:
// 1 coordinate outside +-2^20, 4 no merge because of it or of a box needing more than
// 31 key bits) stay in the workspace header, status_dev = &hdr[0] of its 16 ints.
cudaError_t run_voxel_merge(const mgs_gaussians& in, float voxel, const mgs_merge_params& p,
                            const mgs_gaussians_mut& out, int32_t* partner, int32_t* vox, char* ws_base,
                            cudaStream_t s, int32_t** hdr_dev) {
  MergeWs ws;
  merge_workspace_bytes(in.n, &ws, ws_base);
  if (hdr_dev) *hdr_dev = ws.hdr;
  switch (in.attr_dtype) {
    case MGS_F16: return merge_t<__half>(in, voxel, p, out, partner, vox, ws, s);
    case MGS_BF16: return merge_t<__nv_bfloat16>(in, voxel, p, out, partner, vox, ws, s);
    default: return merge_t<float>(in, voxel, p, out, partner, vox, ws, s);
  }
}

}  // namespace mgs
