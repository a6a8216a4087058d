// FP64 CPU oracle for the MegaParticles hot path (Koide et al., ICRA 2024,
// "Range-based 6-DoF Monte Carlo Localization with GPU-Accelerated Stein
// Particle Filter").
//
// TEST INFRASTRUCTURE ONLY. Nothing on the product path may load this file:
// only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline /
// reference arm call it. It shares no code, header, table or constant
// generator with the CUDA library; the two meet only through the seeded input
// generators and through the definitions written out below.
//
// Style: plain loops, FP64 arithmetic on the FP32 inputs (poses, scan and map
// points as given), std::sort for ordering, brute force or a uniform cell grid
// (an exact candidate filter, pinned against brute force) for radius searches.
// Every function cites the passage of the paper it follows.
//
// Decisions that turn floating point into an integer (a voxel index, a
// neighbour set within a radius, a nearest map point) are taken in FP32 with
// the operation sequences defined in the "FP32 decision sequences" block, so
// that the oracle and the GPU take them in the same precision. All values
// (residuals, information matrices, Hessians, gradients, log-likelihoods,
// SE(3) maps, posteriors) are FP64.
//
// Build: g++ -O2 -std=c++17 -fopenmp -ffp-contract=off -shared -fPIC
// (-ffp-contract=off keeps the un-fused FP32 sequences un-fused; fmaf() is the
// correctly rounded fused multiply-add wherever a sequence says "fused").
//
// Parity pins (tests/test_oracle_*.py) cover every function here; none is
// "parity unpinned".

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <unordered_map>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef int64_t i64;
typedef uint32_t u32;
typedef uint64_t u64;

namespace {

// ---------------------------------------------------------------------------
// Philox-4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw,
// "Parallel random numbers: as easy as 1, 2, 3", SC 2011), written from its
// published definition: ten rounds of two 32x32->64 multiplies with the
// round keys bumped by the Weyl constants between rounds.
// ---------------------------------------------------------------------------
const u32 PHILOX_M0 = 0xD2511F53u, PHILOX_M1 = 0xCD9E8D57u;
const u32 PHILOX_W0 = 0x9E3779B9u, PHILOX_W1 = 0xBB67AE85u;

void philox(const u32 ctr_in[4], const u32 key_in[2], u32 out[4]) {
  u32 c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  u32 k0 = key_in[0], k1 = key_in[1];
  for (int r = 0; r < 10; ++r) {
    u64 p0 = (u64)PHILOX_M0 * (u64)c0;
    u64 p1 = (u64)PHILOX_M1 * (u64)c2;
    u32 hi0 = (u32)(p0 >> 32), lo0 = (u32)p0;
    u32 hi1 = (u32)(p1 >> 32), lo1 = (u32)p1;
    u32 n0 = hi1 ^ c1 ^ k0;
    u32 n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    k0 += PHILOX_W0; k1 += PHILOX_W1;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

// Stream ids (counter word 3) used by the filter.
const u32 STREAM_PREDICT = 1, STREAM_LSH = 2, STREAM_INIT = 3;

// The k-th FP64 uniform in [0,1) of (seed, step, stream): 53 bits from two
// consecutive 32-bit outputs of counter (k/2, 0, step, stream).
double uniform53(u64 seed, u64 step, u32 stream, u32 k) {
  u32 ctr[4] = {k / 2u, 0u, (u32)step, stream};
  u32 key[2] = {(u32)seed, (u32)(seed >> 32)};
  u32 o[4];
  philox(ctr, key, o);
  u32 a = o[2 * (k % 2u)], b = o[2 * (k % 2u) + 1];
  return ((double)(a >> 5) * 67108864.0 + (double)(b >> 6)) / 9007199254740992.0;
}

// A 32-bit output as an open-interval uniform: (x + 1/2) / 2^32.
double uniform32(u32 x) { return ((double)x + 0.5) / 4294967296.0; }

// ---------------------------------------------------------------------------
// SE(3) in FP64. Quaternion q = (x, y, z, w), Hamilton product; twist
// xi = (omega, v), rotation first (the order of W^K, Sec. III-C, Eq. 7);
// right perturbation T exp(xi) (Eq. 1 and Eq. 5).
// ---------------------------------------------------------------------------
struct Quat { double x, y, z, w; };

Quat qmul(const Quat& a, const Quat& b) {
  Quat r;
  r.w = a.w * b.w - a.x * b.x - a.y * b.y - a.z * b.z;
  r.x = a.w * b.x + a.x * b.w + a.y * b.z - a.z * b.y;
  r.y = a.w * b.y - a.x * b.z + a.y * b.w + a.z * b.x;
  r.z = a.w * b.z + a.x * b.y - a.y * b.x + a.z * b.w;
  return r;
}
Quat qconj(const Quat& a) { return Quat{-a.x, -a.y, -a.z, a.w}; }
Quat qnormalize(const Quat& a) {
  double n = std::sqrt(a.x * a.x + a.y * a.y + a.z * a.z + a.w * a.w);
  return Quat{a.x / n, a.y / n, a.z / n, a.w / n};
}

// Rotation matrix of a unit quaternion (row-major).
void quat_to_R(const Quat& q, double R[9]) {
  double x = q.x, y = q.y, z = q.z, w = q.w;
  R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z); R[2] = 2 * (x * z + w * y);
  R[3] = 2 * (x * y + w * z); R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
  R[6] = 2 * (x * z - w * y); R[7] = 2 * (y * z + w * x); R[8] = 1 - 2 * (x * x + y * y);
}

// Quaternion of a rotation matrix (Shepperd's method: branch on the largest
// of the trace and the diagonal).
Quat R_to_quat(const double R[9]) {
  double tr = R[0] + R[4] + R[8];
  Quat q;
  if (tr > R[0] && tr > R[4] && tr > R[8]) {
    double s = std::sqrt(1.0 + tr) * 2;
    q.w = 0.25 * s; q.x = (R[7] - R[5]) / s; q.y = (R[2] - R[6]) / s; q.z = (R[3] - R[1]) / s;
  } else if (R[0] > R[4] && R[0] > R[8]) {
    double s = std::sqrt(1.0 + R[0] - R[4] - R[8]) * 2;
    q.w = (R[7] - R[5]) / s; q.x = 0.25 * s; q.y = (R[1] + R[3]) / s; q.z = (R[2] + R[6]) / s;
  } else if (R[4] > R[8]) {
    double s = std::sqrt(1.0 + R[4] - R[0] - R[8]) * 2;
    q.w = (R[2] - R[6]) / s; q.x = (R[1] + R[3]) / s; q.y = 0.25 * s; q.z = (R[5] + R[7]) / s;
  } else {
    double s = std::sqrt(1.0 + R[8] - R[0] - R[4]) * 2;
    q.w = (R[3] - R[1]) / s; q.x = (R[2] + R[6]) / s; q.y = (R[5] + R[7]) / s; q.z = 0.25 * s;
  }
  if (q.w < 0) { q.x = -q.x; q.y = -q.y; q.z = -q.z; q.w = -q.w; }
  return qnormalize(q);
}

void matvec3(const double M[9], const double v[3], double o[3]) {
  for (int r = 0; r < 3; ++r) o[r] = M[3 * r] * v[0] + M[3 * r + 1] * v[1] + M[3 * r + 2] * v[2];
}
void matTvec3(const double M[9], const double v[3], double o[3]) {
  for (int r = 0; r < 3; ++r) o[r] = M[r] * v[0] + M[3 + r] * v[1] + M[6 + r] * v[2];
}
void skew(const double v[3], double S[9]) {
  S[0] = 0; S[1] = -v[2]; S[2] = v[1];
  S[3] = v[2]; S[4] = 0; S[5] = -v[0];
  S[6] = -v[1]; S[7] = v[0]; S[8] = 0;
}
void matmul3(const double A[9], const double B[9], double C[9]) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0;
      for (int k = 0; k < 3; ++k) s += A[3 * i + k] * B[3 * k + j];
      C[3 * i + j] = s;
    }
}

// exp: so(3) -> unit quaternion.
Quat so3_exp(const double w[3]) {
  double th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
  double th = std::sqrt(th2);
  double s, c;
  if (th < 1e-5) {
    s = 0.5 - th2 / 48.0;          // sin(th/2)/th
    c = 1.0 - th2 / 8.0;           // cos(th/2)
  } else {
    s = std::sin(0.5 * th) / th;
    c = std::cos(0.5 * th);
  }
  return Quat{s * w[0], s * w[1], s * w[2], c};
}

// log: unit quaternion -> so(3), angle in [0, pi].
void so3_log(Quat q, double w[3]) {
  if (q.w < 0) { q.x = -q.x; q.y = -q.y; q.z = -q.z; q.w = -q.w; }
  double s = std::sqrt(q.x * q.x + q.y * q.y + q.z * q.z);
  double f;
  if (s < 1e-10) {
    f = 2.0 / q.w * (1.0 - s * s / (3.0 * q.w * q.w));
  } else {
    f = 2.0 * std::atan2(s, q.w) / s;
  }
  w[0] = f * q.x; w[1] = f * q.y; w[2] = f * q.z;
}

// Left Jacobian V(w) = I + A [w]x + B [w]x^2 and its inverse
// V^-1(w) = I - 1/2 [w]x + C [w]x^2.
void V_of(const double w[3], double V[9], bool inverse) {
  double th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
  double th = std::sqrt(th2);
  double S[9], S2[9];
  skew(w, S);
  matmul3(S, S, S2);
  // Evaluated without cancellation: A = 2 sin^2(th/2) / th^2,
  // B = (th - sin th) / th^3 and C = (1 - (th/2) cot(th/2)) / th^2, with their
  // Taylor series below th = 1e-2.
  double a, b;
  if (!inverse) {
    if (th < 1e-2) {
      a = 0.5 - th2 / 24.0 + th2 * th2 / 720.0;
      b = 1.0 / 6.0 - th2 / 120.0 + th2 * th2 / 5040.0;
    } else {
      double sh = std::sin(0.5 * th);
      a = 2.0 * sh * sh / th2;
      b = (th - std::sin(th)) / (th2 * th);
    }
  } else {
    a = -0.5;
    if (th < 1e-2) b = 1.0 / 12.0 + th2 / 720.0 + th2 * th2 / 30240.0;
    else {
      double h = 0.5 * th;
      b = (1.0 - h * std::cos(h) / std::sin(h)) / th2;
    }
  }
  for (int i = 0; i < 9; ++i) V[i] = a * S[i] + b * S2[i];
  V[0] += 1; V[4] += 1; V[8] += 1;
}

struct Pose { Quat q; double t[3]; };

Pose se3_exp(const double xi[6]) {
  Pose P;
  P.q = so3_exp(xi);
  double V[9];
  V_of(xi, V, false);
  matvec3(V, xi + 3, P.t);
  return P;
}

void se3_log(const Pose& P, double xi[6]) {
  so3_log(P.q, xi);
  double Vi[9];
  V_of(xi, Vi, true);
  matvec3(Vi, P.t, xi + 3);
}

Pose compose(const Pose& A, const Pose& B) {
  Pose C;
  C.q = qmul(A.q, B.q);
  double R[9], Rt[3];
  quat_to_R(qnormalize(A.q), R);
  matvec3(R, B.t, Rt);
  for (int i = 0; i < 3; ++i) C.t[i] = Rt[i] + A.t[i];
  return C;
}

Pose inverse(const Pose& A) {
  Pose B;
  B.q = qconj(A.q);
  double R[9];
  quat_to_R(qnormalize(A.q), R);
  double mt[3];
  matTvec3(R, A.t, mt);
  for (int i = 0; i < 3; ++i) B.t[i] = -mt[i];
  return B;
}

// A stored particle pose: FP32 (qx, qy, qz, qw, tx, ty, tz), read in FP64 and
// normalised in FP64 for the SE(3) operations.
Pose pose_from_f32(const float* p) {
  Pose P;
  P.q = qnormalize(Quat{(double)p[0], (double)p[1], (double)p[2], (double)p[3]});
  P.t[0] = p[4]; P.t[1] = p[5]; P.t[2] = p[6];
  return P;
}

// d_ij = log(T_i^-1 T_j), Eq. 8.
void relative_log(const Pose& Ti, const Pose& Tj, double d[6]) {
  Pose r = compose(inverse(Ti), Tj);
  se3_log(r, d);
}

// ---------------------------------------------------------------------------
// FP32 decision sequences. Each operation is rounded to FP32; "fused" marks a
// single-rounding fused multiply-add (fmaf). These are the only places where
// the oracle follows FP32 arithmetic, and only to take integer decisions.
// ---------------------------------------------------------------------------
// (D1) rotation of a stored quaternion, un-fused.
void R32_of(const float* q, float R[9]) {
  float x = q[0], y = q[1], z = q[2], w = q[3];
  float x2 = x + x, y2 = y + y, z2 = z + z;
  float xx = x * x2, yy = y * y2, zz = z * z2;
  float xy = x * y2, xz = x * z2, yz = y * z2;
  float wx = w * x2, wy = w * y2, wz = w * z2;
  R[0] = 1.0f - (yy + zz); R[1] = xy - wz; R[2] = xz + wy;
  R[3] = xy + wz; R[4] = 1.0f - (xx + zz); R[5] = yz - wx;
  R[6] = xz - wy; R[7] = yz + wx; R[8] = 1.0f - (xx + yy);
}
// (D2) transformed scan point q = R mu + t: qt_a = fused(R_a2, mu_z,
// fused(R_a1, mu_y, R_a0 * mu_x)); q_a = qt_a + t_a.
void transform32(const float R[9], const float* t, const float* mu, float q[3]) {
  for (int a = 0; a < 3; ++a) {
    float qt = fmaf(R[3 * a + 2], mu[2], fmaf(R[3 * a + 1], mu[1], R[3 * a] * mu[0]));
    q[a] = qt + t[a];
  }
}
// (D3) squared distance ((dx*dx + dy*dy) + dz*dz), dx = b_x - a_x, un-fused.
float dist2_32(const float* a, const float* b) {
  float dx = b[0] - a[0], dy = b[1] - a[1], dz = b[2] - a[2];
  float s = dx * dx;
  float s2 = dy * dy;
  s = s + s2;
  float s3 = dz * dz;
  return s + s3;
}

// (D4) NNF grid geometry from the valid map points: lo/hi = exact FP32
// min/max; o = lo - r_max; n = floor(((hi + r_max) - o) * inv_res) + 1;
// inv_res = 1/res (FP32 division); off = -(o * inv_res).
struct Grid {
  float o[3];
  int n[3];
  float res, inv_res, off[3];
};
Grid grid_geometry(const float* pts, i64 n, const uint8_t* valid, float res, float r_max) {
  float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (i64 i = 0; i < n; ++i) {
    if (valid && !valid[i]) continue;
    for (int a = 0; a < 3; ++a) {
      lo[a] = std::min(lo[a], pts[3 * i + a]);
      hi[a] = std::max(hi[a], pts[3 * i + a]);
    }
  }
  Grid g;
  g.res = res;
  g.inv_res = 1.0f / res;
  for (int a = 0; a < 3; ++a) {
    g.o[a] = lo[a] - r_max;
    float t1 = hi[a] + r_max;
    float t2 = t1 - g.o[a];
    float t3 = t2 * g.inv_res;
    g.n[a] = (int)std::floor(t3) + 1;
    float p = g.o[a] * g.inv_res;
    g.off[a] = -p;
  }
  return g;
}
// (D5) voxel coordinate v_a = floor(fused(q_a, inv_res, off_a)).
void voxel_of(const Grid& g, const float q[3], int v[3]) {
  for (int a = 0; a < 3; ++a) v[a] = (int)std::floor(fmaf(q[a], g.inv_res, g.off[a]));
}
bool inside(const Grid& g, const int v[3]) {
  return v[0] >= 0 && v[1] >= 0 && v[2] >= 0 && v[0] < g.n[0] && v[1] < g.n[1] && v[2] < g.n[2];
}
// (D6) voxel centre c_a = o_a + ((float)v_a + 0.5) * res.
void voxel_centre(const Grid& g, const int v[3], float c[3]) {
  for (int a = 0; a < 3; ++a) {
    float h = (float)v[a] + 0.5f;
    float m = h * g.res;
    c[a] = g.o[a] + m;
  }
}

// ---------------------------------------------------------------------------
// Exact radius search helper: a uniform cell grid of side h (FP64), used only
// to skip points that cannot be within the radius; the decision itself is the
// FP32 distance test. h exceeds the radius by 1e-5 relative so that every
// point whose FP32 distance passes lies in the 27 cells around the query.
// Pinned against brute force by the tests.
// ---------------------------------------------------------------------------
struct CellGrid {
  double h, o[3];
  int n[3];
  std::vector<i64> start;   // size ncell + 1
  std::vector<i64> items;   // point ids in increasing order within a cell
  void build(const float* pts, i64 n_pts, const uint8_t* valid, double radius) {
    h = radius * (1.0 + 1e-5);
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (i64 i = 0; i < n_pts; ++i) {
      if (valid && !valid[i]) continue;
      for (int a = 0; a < 3; ++a) { lo[a] = std::min(lo[a], (double)pts[3 * i + a]); hi[a] = std::max(hi[a], (double)pts[3 * i + a]); }
    }
    if (lo[0] > hi[0]) { for (int a = 0; a < 3; ++a) { lo[a] = 0; hi[a] = 0; } }
    for (int a = 0; a < 3; ++a) { o[a] = lo[a] - h; n[a] = (int)std::floor((hi[a] - o[a]) / h) + 2; }
    i64 nc = (i64)n[0] * n[1] * n[2];
    std::vector<i64> cnt(nc + 1, 0);
    std::vector<i64> cell_of(n_pts, -1);
    for (i64 i = 0; i < n_pts; ++i) {
      if (valid && !valid[i]) continue;
      i64 c = cell_index(pts + 3 * i);
      cell_of[i] = c;
      cnt[c + 1]++;
    }
    for (i64 c = 0; c < nc; ++c) cnt[c + 1] += cnt[c];
    start = cnt;
    items.assign(cnt[nc], 0);
    std::vector<i64> fill(cnt.begin(), cnt.end() - 1);
    for (i64 i = 0; i < n_pts; ++i)
      if (cell_of[i] >= 0) items[fill[cell_of[i]]++] = i;
  }
  void cell_coords(const float* p, int c[3]) const {
    for (int a = 0; a < 3; ++a) {
      int v = (int)std::floor(((double)p[a] - o[a]) / h);
      c[a] = std::min(std::max(v, -1), n[a]);
    }
  }
  i64 cell_index(const float* p) const {
    int c[3];
    cell_coords(p, c);
    return ((i64)c[2] * n[1] + c[1]) * n[0] + c[0];
  }
  // Calls f(id) for every point in the 27 cells around p.
  template <class F> void visit(const float* p, F f) const {
    int c[3];
    cell_coords(p, c);
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          int x = c[0] + dx, y = c[1] + dy, z = c[2] + dz;
          if (x < 0 || y < 0 || z < 0 || x >= n[0] || y >= n[1] || z >= n[2]) continue;
          i64 ci = ((i64)z * n[1] + y) * n[0] + x;
          for (i64 k = start[ci]; k < start[ci + 1]; ++k) f(items[k]);
        }
  }
};

// ---------------------------------------------------------------------------
// Symmetric 3x3 eigen-decomposition by cyclic Jacobi rotations (FP64).
// Eigenvalues ascending; eigenvectors are the columns of V.
// ---------------------------------------------------------------------------
void sym3_eigh(const double Ain[9], double w[3], double V[9]) {
  double A[3][3];
  double Q[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) A[i][j] = 0.5 * (Ain[3 * i + j] + Ain[3 * j + i]);
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2];
    double scale = A[0][0] * A[0][0] + A[1][1] * A[1][1] + A[2][2] * A[2][2] + 2 * off;
    if (off <= 1e-32 * scale || off == 0.0) break;
    for (int p = 0; p < 2; ++p)
      for (int q = p + 1; q < 3; ++q) {
        if (A[p][q] == 0.0) continue;
        double theta = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
        double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < 3; ++k) {  // A <- A J
          double akp = A[k][p], akq = A[k][q];
          A[k][p] = c * akp - s * akq;
          A[k][q] = s * akp + c * akq;
        }
        for (int k = 0; k < 3; ++k) {  // A <- J^T A
          double apk = A[p][k], aqk = A[q][k];
          A[p][k] = c * apk - s * aqk;
          A[q][k] = s * apk + c * aqk;
        }
        for (int k = 0; k < 3; ++k) {  // Q <- Q J
          double qkp = Q[k][p], qkq = Q[k][q];
          Q[k][p] = c * qkp - s * qkq;
          Q[k][q] = s * qkp + c * qkq;
        }
      }
  }
  int idx[3] = {0, 1, 2};
  std::sort(idx, idx + 3, [&](int a, int b) { return A[a][a] < A[b][b] || (A[a][a] == A[b][b] && a < b); });
  for (int c = 0; c < 3; ++c) {
    w[c] = A[idx[c]][idx[c]];
    for (int r = 0; r < 3; ++r) V[3 * r + c] = Q[r][idx[c]];
  }
}

// 3x3 inverse by the adjugate (FP64).
bool inv3(const double M[9], double I[9]) {
  double c00 = M[4] * M[8] - M[5] * M[7];
  double c01 = M[5] * M[6] - M[3] * M[8];
  double c02 = M[3] * M[7] - M[4] * M[6];
  double det = M[0] * c00 + M[1] * c01 + M[2] * c02;
  if (!(std::fabs(det) > 0)) return false;
  double id = 1.0 / det;
  I[0] = c00 * id; I[1] = (M[2] * M[7] - M[1] * M[8]) * id; I[2] = (M[1] * M[5] - M[2] * M[4]) * id;
  I[3] = c01 * id; I[4] = (M[0] * M[8] - M[2] * M[6]) * id; I[5] = (M[2] * M[3] - M[0] * M[5]) * id;
  I[6] = c02 * id; I[7] = (M[1] * M[6] - M[0] * M[7]) * id; I[8] = (M[0] * M[4] - M[1] * M[3]) * id;
  return true;
}

// GICP covariance of a point with normal n: eigenvalues (1, 1, eps) with n the
// eigenvector of eps, i.e. Sigma = I - (1 - eps) n n^T (Sec. III-C, "each
// point modelled as a Gaussian"; regularisation of Segal et al. 2009).
void gicp_cov(const double n[3], double eps, double S[9]) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) S[3 * i + j] = (i == j ? 1.0 : 0.0) - (1.0 - eps) * n[i] * n[j];
}

const int H_IDX[6][6] = {
    {0, 1, 2, 3, 4, 5}, {1, 6, 7, 8, 9, 10}, {2, 7, 11, 12, 13, 14},
    {3, 8, 12, 15, 16, 17}, {4, 9, 13, 16, 18, 19}, {5, 10, 14, 17, 19, 20}};

// ---------------------------------------------------------------------------
// Map object: valid map points with normals, NNF grid geometry, exact radius
// search grid.
// ---------------------------------------------------------------------------
struct Map {
  std::vector<float> pts;
  std::vector<uint8_t> valid;
  std::vector<double> normals;
  i64 n = 0;
  Grid g;
  float r_max = 0, r2 = 0;
  CellGrid cells;
};

// NNF value of voxel v (Sec. III-C, nearest neighbour field): the valid map
// point nearest to the voxel centre by (D3), among those with distance^2 <=
// r_max^2 (FP32), ties to the smaller index; -1 if none.
int nnf_value(const Map& M, const int v[3], bool brute) {
  float c[3];
  voxel_centre(M.g, v, c);
  int best = -1;
  float bd = 0;
  auto consider = [&](i64 j) {
    float d2 = dist2_32(c, &M.pts[3 * j]);
    if (!(d2 <= M.r2)) return;
    if (best < 0 || d2 < bd || (d2 == bd && j < best)) { best = (int)j; bd = d2; }
  };
  if (brute) {
    for (i64 j = 0; j < M.n; ++j) if (M.valid[j]) consider(j);
  } else {
    M.cells.visit(c, consider);
  }
  return best;
}

}  // namespace

extern "C" {

int or_version() { return 1; }

void or_philox4x32_10(const u32 ctr[4], const u32 key[2], u32 out[4]) { philox(ctr, key, out); }

double or_uniform53(u64 seed, u64 step, u32 stream, u32 k) { return uniform53(seed, step, stream, k); }

// ---- SE(3) (Sec. III-B Eq. 1, Sec. III-C Eq. 5 and Eq. 8) ----
void or_quat_to_rot(const double q[4], double R[9]) { quat_to_R(qnormalize(Quat{q[0], q[1], q[2], q[3]}), R); }

void or_rot_to_quat(const double R[9], double q[4]) {
  Quat Q = R_to_quat(R);
  q[0] = Q.x; q[1] = Q.y; q[2] = Q.z; q[3] = Q.w;
}

void or_se3_exp(const double xi[6], double q[4], double t[3]) {
  Pose P = se3_exp(xi);
  q[0] = P.q.x; q[1] = P.q.y; q[2] = P.q.z; q[3] = P.q.w;
  t[0] = P.t[0]; t[1] = P.t[1]; t[2] = P.t[2];
}

void or_se3_log(const double q[4], const double t[3], double xi[6]) {
  Pose P;
  P.q = qnormalize(Quat{q[0], q[1], q[2], q[3]});
  P.t[0] = t[0]; P.t[1] = t[1]; P.t[2] = t[2];
  se3_log(P, xi);
}

// d = log(Ti^-1 Tj) for FP32 stored poses (Eq. 8).
void or_relative_log(const float* pi, const float* pj, double d[6]) {
  relative_log(pose_from_f32(pi), pose_from_f32(pj), d);
}

int or_sym3_eigh(const double A[9], double w[3], double V[9]) {
  sym3_eigh(A, w, V);
  return 0;
}

// ---- Point Gaussians (Sec. III-C, "Likelihood evaluation") ----
// For each point i: the up-to-k nearest points (itself included) among those
// with FP32 distance^2 (D3) <= r_cov^2, ordered by (distance^2, index). With
// fewer than kmin such points the point is invalid. Otherwise the sample
// covariance of the neighbourhood (FP64) gives the normal = eigenvector of its
// smallest eigenvalue, sign fixed so that its largest-magnitude component is
// positive (the covariance I - (1-eps) n n^T does not depend on the sign).
int or_point_normals(const float* pts, i64 n, float r_cov, int k, int kmin, int brute,
                     double* normals, uint8_t* valid, int32_t* nbrs, double* covs, int nthreads) {
  float r2 = r_cov * r_cov;
  CellGrid cg;
  if (!brute) cg.build(pts, n, nullptr, (double)r_cov);
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 256)
#endif
  for (i64 i = 0; i < n; ++i) {
    std::vector<std::pair<float, i64>> cand;
    auto consider = [&](i64 j) {
      float d2 = dist2_32(&pts[3 * i], &pts[3 * j]);
      if (d2 <= r2) cand.push_back({d2, j});
    };
    if (brute) { for (i64 j = 0; j < n; ++j) consider(j); }
    else cg.visit(&pts[3 * i], consider);
    std::sort(cand.begin(), cand.end());
    int m = std::min<int>((int)cand.size(), k);
    if (nbrs) for (int a = 0; a < k; ++a) nbrs[i * k + a] = a < m ? (int32_t)cand[a].second : -1;
    if (m < kmin) {
      valid[i] = 0;
      normals[3 * i] = normals[3 * i + 1] = normals[3 * i + 2] = 0;
      if (covs) for (int a = 0; a < 9; ++a) covs[9 * i + a] = 0;
      continue;
    }
    double mean[3] = {0, 0, 0};
    for (int a = 0; a < m; ++a)
      for (int c = 0; c < 3; ++c) mean[c] += pts[3 * cand[a].second + c];
    for (int c = 0; c < 3; ++c) mean[c] /= m;
    double C[9] = {0};
    for (int a = 0; a < m; ++a) {
      double d[3];
      for (int c = 0; c < 3; ++c) d[c] = pts[3 * cand[a].second + c] - mean[c];
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) C[3 * r + c] += d[r] * d[c];
    }
    for (int a = 0; a < 9; ++a) C[a] /= m;
    if (covs) for (int a = 0; a < 9; ++a) covs[9 * i + a] = C[a];
    double w[3], V[9];
    sym3_eigh(C, w, V);
    double nv[3] = {V[0], V[3], V[6]};
    int big = 0;
    for (int c = 1; c < 3; ++c) if (std::fabs(nv[c]) > std::fabs(nv[big])) big = c;
    double sgn = nv[big] < 0 ? -1.0 : 1.0;
    double nn = std::sqrt(nv[0] * nv[0] + nv[1] * nv[1] + nv[2] * nv[2]);
    for (int c = 0; c < 3; ++c) normals[3 * i + c] = sgn * nv[c] / nn;
    valid[i] = 1;
  }
  return 0;
}

// ---- Map / NNF (Sec. III-C, nearest neighbour field m^nnf) ----
void* or_map_create(const float* pts, i64 n, const uint8_t* valid, const double* normals, float res, float r_max) {
  Map* M = new Map();
  M->n = n;
  M->pts.assign(pts, pts + 3 * n);
  M->valid.assign(valid, valid + n);
  M->normals.assign(normals, normals + 3 * n);
  M->g = grid_geometry(pts, n, valid, res, r_max);
  M->r_max = r_max;
  M->r2 = r_max * r_max;
  M->cells.build(pts, n, valid, (double)r_max);
  return M;
}

void or_map_destroy(void* h) { delete (Map*)h; }

void or_map_geometry(void* h, float origin[3], int32_t dims[3], float* inv_res, float off[3]) {
  Map* M = (Map*)h;
  for (int a = 0; a < 3; ++a) { origin[a] = M->g.o[a]; dims[a] = M->g.n[a]; off[a] = M->g.off[a]; }
  *inv_res = M->g.inv_res;
}

void or_map_nnf(void* h, const int32_t* vox, i64 m, int32_t* out, int brute, int nthreads) {
  Map* M = (Map*)h;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 64)
#endif
  for (i64 i = 0; i < m; ++i) {
    int v[3] = {vox[3 * i], vox[3 * i + 1], vox[3 * i + 2]};
    out[i] = inside(M->g, v) ? nnf_value(*M, v, brute != 0) : -1;
  }
}

// Voxel of a scan point under a stored pose, by (D1), (D2), (D5).
void or_voxel_of(void* h, const float* pose, const float* mu, int32_t v[3], float q_out[3]) {
  Map* M = (Map*)h;
  float R[9];
  R32_of(pose, R);
  float q[3];
  transform32(R, pose + 4, mu, q);
  int vv[3];
  voxel_of(M->g, q, vv);
  for (int a = 0; a < 3; ++a) { v[a] = vv[a]; q_out[a] = q[a]; }
}

// ---- Likelihood and Gauss-Newton terms (Sec. III-C Eq. 2, 3, 4) ----
// For particle T = (R, t) and each valid scan point k:
//   correspondence m = NNF[voxel(T mu_k)] (FP32 decision, -1 if outside);
//   e_k = mu^M_m - T mu^S_k;  Omega_k = (Sigma^M_m + R Sigma^S_k R^T)^-1;
//   c_k = e_k^T Omega_k e_k;  inlier iff m >= 0 and c_k <= c_max;
//   log p -= inlier ? c_k : c_max   (truncated quadratic);
//   for inliers, J_k = d e_k / d xi = R [ [mu^S_k]x , -I ]  (right
//   perturbation T exp(xi)), H += J^T Omega J, b += J^T Omega e.
// amb counts inlier decisions within amb_tol * c_max of the threshold.
// absum (optional, np x 28): per output entry the sum of the magnitudes of
// its terms (H 21, b 6, log-likelihood 1), the scale of its rounding error.
// ambabs (optional, np x 28): the same sums over the ambiguous pairs only
// (for the log-likelihood: |c_k - c_max|), i.e. how far an output can move if
// an implementation in another precision takes the other inlier decision.
int or_likelihood(void* h, const float* poses, i64 np, const float* scan, const double* scan_n,
                  const uint8_t* scan_valid, i64 ns, double c_max, double eps_cov, double amb_tol,
                  double* H, double* b, double* loglik, int32_t* n_in, int32_t* amb, double* absum,
                  double* ambabs, int nthreads) {
  Map* M = (Map*)h;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
#endif
  {
    std::unordered_map<i64, int> memo;
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 4)
#endif
    for (i64 i = 0; i < np; ++i) {
      const float* P = poses + 7 * i;
      float R32[9];
      R32_of(P, R32);
      Quat q{(double)P[0], (double)P[1], (double)P[2], (double)P[3]};
      double R[9];
      quat_to_R(q, R);  // the stored quaternion as given (unit up to FP32 rounding)
      double t[3] = {P[4], P[5], P[6]};
      double Hl[21] = {0}, bl[6] = {0}, ll = 0, ab[28] = {0}, aa[28] = {0};
      int cnt = 0, namb = 0;
      for (i64 k = 0; k < ns; ++k) {
        if (scan_valid && !scan_valid[k]) continue;
        const float* mu = scan + 3 * k;
        float q32[3];
        transform32(R32, P + 4, mu, q32);
        int v[3];
        voxel_of(M->g, q32, v);
        int m = -1;
        if (inside(M->g, v)) {
          i64 lin = ((i64)v[2] * M->g.n[1] + v[1]) * M->g.n[0] + v[0];
          auto it = memo.find(lin);
          if (it != memo.end()) m = it->second;
          else { m = nnf_value(*M, v, false); memo.emplace(lin, m); }
        }
        if (m < 0) { ll -= c_max; ab[27] += c_max; continue; }
        double mus[3] = {mu[0], mu[1], mu[2]};
        double qk[3];
        matvec3(R, mus, qk);
        for (int a = 0; a < 3; ++a) qk[a] += t[a];
        double e[3];
        for (int a = 0; a < 3; ++a) e[a] = (double)M->pts[3 * m + a] - qk[a];
        double SM[9], SS[9], RS[9], RSRt[9], Rt[9], C[9], Om[9];
        gicp_cov(&M->normals[3 * m], eps_cov, SM);
        gicp_cov(scan_n + 3 * k, eps_cov, SS);
        for (int r = 0; r < 3; ++r) for (int c = 0; c < 3; ++c) Rt[3 * r + c] = R[3 * c + r];
        matmul3(R, SS, RS);
        matmul3(RS, Rt, RSRt);
        for (int a = 0; a < 9; ++a) C[a] = SM[a] + RSRt[a];
        if (!inv3(C, Om)) { ll -= c_max; ab[27] += c_max; continue; }
        double Oe[3];
        matvec3(Om, e, Oe);
        double c = e[0] * Oe[0] + e[1] * Oe[1] + e[2] * Oe[2];
        const bool near = std::fabs(c - c_max) <= amb_tol * c_max;
        const bool inl = c <= c_max;
        if (near) { namb++; aa[27] += std::fabs(c - c_max); }
        if (!inl) {
          ll -= c_max;
          ab[27] += c_max;
          if (!near) continue;
        } else {
          ll -= c;
          ab[27] += std::fabs(c);
          cnt++;
        }
        // J = R [ [mu]x , -I ]
        double S[9], J0[9], J[3][6];
        skew(mus, S);
        matmul3(R, S, J0);
        for (int r = 0; r < 3; ++r)
          for (int c2 = 0; c2 < 3; ++c2) { J[r][c2] = J0[3 * r + c2]; J[r][3 + c2] = -R[3 * r + c2]; }
        double OJ[3][6];
        for (int r = 0; r < 3; ++r)
          for (int c2 = 0; c2 < 6; ++c2) OJ[r][c2] = Om[3 * r] * J[0][c2] + Om[3 * r + 1] * J[1][c2] + Om[3 * r + 2] * J[2][c2];
        for (int a = 0; a < 6; ++a) {
          for (int bb = a; bb < 6; ++bb) {
            double s = 0;
            for (int r = 0; r < 3; ++r) s += J[r][a] * OJ[r][bb];
            if (inl) {
              Hl[H_IDX[a][bb]] += s;
              ab[H_IDX[a][bb]] += std::fabs(s);
            }
            if (near) aa[H_IDX[a][bb]] += std::fabs(s);
          }
          double s = 0;
          for (int r = 0; r < 3; ++r) s += J[r][a] * Oe[r];
          if (inl) {
            bl[a] += s;
            ab[21 + a] += std::fabs(s);
          }
          if (near) aa[21 + a] += std::fabs(s);
        }
      }
      for (int a = 0; a < 21; ++a) H[21 * i + a] = Hl[a];
      for (int a = 0; a < 6; ++a) b[6 * i + a] = bl[a];
      loglik[i] = ll;
      n_in[i] = cnt;
      if (amb) amb[i] = namb;
      if (absum) for (int a = 0; a < 28; ++a) absum[28 * i + a] = ab[a];
      if (ambabs) for (int a = 0; a < 28; ++a) ambabs[28 * i + a] = aa[a];
    }
  }
  return 0;
}

// Per-pair dump for one particle (for finite-difference pins): m, e, Omega, J,
// c and the inlier flag of every scan point (invalid scan points: m = -2).
int or_likelihood_pairs(void* h, const float* pose, const float* scan, const double* scan_n,
                        const uint8_t* scan_valid, i64 ns, double c_max, double eps_cov,
                        int32_t* m_out, double* e_out, double* om_out, double* J_out, double* c_out,
                        uint8_t* inl_out) {
  Map* M = (Map*)h;
  float R32[9];
  R32_of(pose, R32);
  double R[9];
  quat_to_R(Quat{(double)pose[0], (double)pose[1], (double)pose[2], (double)pose[3]}, R);
  double t[3] = {pose[4], pose[5], pose[6]};
  for (i64 k = 0; k < ns; ++k) {
    for (int a = 0; a < 3; ++a) e_out[3 * k + a] = 0;
    for (int a = 0; a < 9; ++a) om_out[9 * k + a] = 0;
    for (int a = 0; a < 18; ++a) J_out[18 * k + a] = 0;
    c_out[k] = 0; inl_out[k] = 0;
    if (scan_valid && !scan_valid[k]) { m_out[k] = -2; continue; }
    const float* mu = scan + 3 * k;
    float q32[3];
    transform32(R32, pose + 4, mu, q32);
    int v[3];
    voxel_of(M->g, q32, v);
    int m = inside(M->g, v) ? nnf_value(*M, v, false) : -1;
    m_out[k] = m;
    if (m < 0) continue;
    double mus[3] = {mu[0], mu[1], mu[2]}, qk[3];
    matvec3(R, mus, qk);
    for (int a = 0; a < 3; ++a) e_out[3 * k + a] = (double)M->pts[3 * m + a] - (qk[a] + t[a]);
    double SM[9], SS[9], RS[9], RSRt[9], Rt[9], C[9], Om[9];
    gicp_cov(&M->normals[3 * m], eps_cov, SM);
    gicp_cov(scan_n + 3 * k, eps_cov, SS);
    for (int r = 0; r < 3; ++r) for (int c = 0; c < 3; ++c) Rt[3 * r + c] = R[3 * c + r];
    matmul3(R, SS, RS);
    matmul3(RS, Rt, RSRt);
    for (int a = 0; a < 9; ++a) C[a] = SM[a] + RSRt[a];
    inv3(C, Om);
    for (int a = 0; a < 9; ++a) om_out[9 * k + a] = Om[a];
    double Oe[3];
    matvec3(Om, e_out + 3 * k, Oe);
    double c = 0;
    for (int a = 0; a < 3; ++a) c += e_out[3 * k + a] * Oe[a];
    c_out[k] = c;
    inl_out[k] = c <= c_max ? 1 : 0;
    double S[9], J0[9];
    skew(mus, S);
    matmul3(R, S, J0);
    for (int r = 0; r < 3; ++r)
      for (int c2 = 0; c2 < 3; ++c2) { J_out[18 * k + 6 * r + c2] = J0[3 * r + c2]; J_out[18 * k + 6 * r + 3 + c2] = -R[3 * r + c2]; }
  }
  return 0;
}

// ---- Gauss-Newton displacement (Sec. III-C, psi = H^-1 b, Eq. 4) ----
// psi = -(H + lambda diag(H) + eps I)^-1 b by an LDL^T factorisation (FP64);
// psi = 0 when fewer than 6 inliers or a pivot is not positive. The minus
// sign makes psi the step that increases log p under J = d e / d xi.
void or_gn_solve(const double* H, const double* b, const int32_t* n_in, i64 np, double lambda,
                 double eps, double* psi, int32_t* ok) {
  for (i64 i = 0; i < np; ++i) {
    double A[6][6];
    for (int r = 0; r < 6; ++r)
      for (int c = 0; c < 6; ++c) A[r][c] = H[21 * i + H_IDX[r][c]];
    for (int r = 0; r < 6; ++r) A[r][r] += lambda * A[r][r] + eps;
    double L[6][6] = {{0}}, D[6];
    bool good = n_in[i] >= 6;
    for (int j = 0; j < 6 && good; ++j) {
      double d = A[j][j];
      for (int k = 0; k < j; ++k) d -= L[j][k] * L[j][k] * D[k];
      if (!(d > 0)) { good = false; break; }
      D[j] = d;
      L[j][j] = 1;
      for (int r = j + 1; r < 6; ++r) {
        double s = A[r][j];
        for (int k = 0; k < j; ++k) s -= L[r][k] * L[j][k] * D[k];
        L[r][j] = s / d;
      }
    }
    double x[6] = {0};
    if (good) {
      double y[6];
      for (int r = 0; r < 6; ++r) {
        double s = -b[6 * i + r];
        for (int k = 0; k < r; ++k) s -= L[r][k] * y[k];
        y[r] = s;
      }
      for (int r = 0; r < 6; ++r) y[r] /= D[r];
      for (int r = 5; r >= 0; --r) {
        double s = y[r];
        for (int k = r + 1; k < 6; ++k) s -= L[k][r] * x[k];
        x[r] = s;
      }
    }
    for (int r = 0; r < 6; ++r) psi[6 * i + r] = x[r];
    if (ok) ok[i] = good ? 1 : 0;
  }
}

// ---- LSH (Sec. III-C Eq. 9 and Eq. 10, Algorithm 1) ----
// T^LSH and delta^LSH for one step, drawn in FP64 from Philox(seed) with
// counter (k/2, 0, step, STREAM_LSH): uniforms u0..u2 give a uniform rotation
// (Shoemake), u3..u5 a translation uniform in [lo, hi], u6..u11 three
// Box-Muller pairs scaled by sigma.
void or_lsh_draw(u64 seed, u64 step, const double lo[3], const double hi[3], double sigma,
                 double q[4], double t[3], double delta[6]) {
  double u[12];
  for (u32 k = 0; k < 12; ++k) u[k] = uniform53(seed, step, STREAM_LSH, k);
  const double two_pi = 6.283185307179586476925286766559;
  double a = std::sqrt(1.0 - u[0]), bq = std::sqrt(u[0]);
  q[0] = a * std::sin(two_pi * u[1]);
  q[1] = a * std::cos(two_pi * u[1]);
  q[2] = bq * std::sin(two_pi * u[2]);
  q[3] = bq * std::cos(two_pi * u[2]);
  for (int c = 0; c < 3; ++c) t[c] = lo[c] + u[3 + c] * (hi[c] - lo[c]);
  for (int p = 0; p < 3; ++p) {
    double r = std::sqrt(-2.0 * std::log(1.0 - u[6 + 2 * p]));
    double th = two_pi * u[7 + 2 * p];
    delta[2 * p] = sigma * r * std::cos(th);
    delta[2 * p + 1] = sigma * r * std::sin(th);
  }
}

// zeta = alpha W^K log(T_LSH^-1 T_i) + delta (Eq. 10, FP64); c_a = floor(zeta_a);
// key = XOR_a (c_a * P_a) mod 2^32 (the tuple hash of Teschner et al. 2003
// extended to six components); bucket = key mod 2^nb_log2. flags = 1 when a
// zeta_a lies within 1e-9 of an integer.
void or_lsh_keys(const float* poses, i64 np, const double q[4], const double t[3], const double delta[6],
                 double alpha, double sr, double st, int nb_log2, u32* keys, u32* buckets, int32_t* flags,
                 double* zeta_out) {
  static const u32 P[6] = {73856093u, 19349663u, 83492791u, 2654435761u, 805459861u, 3674653429u};
  Pose L;
  L.q = qnormalize(Quat{q[0], q[1], q[2], q[3]});
  L.t[0] = t[0]; L.t[1] = t[1]; L.t[2] = t[2];
  Pose Li = inverse(L);
  double W[6] = {sr, sr, sr, st, st, st};
  for (i64 i = 0; i < np; ++i) {
    Pose Ti = pose_from_f32(poses + 7 * i);
    double d[6];
    se3_log(compose(Li, Ti), d);
    u32 key = 0;
    int fl = 0;
    for (int a = 0; a < 6; ++a) {
      double z = alpha * W[a] * d[a] + delta[a];
      if (zeta_out) zeta_out[6 * i + a] = z;
      double f = std::floor(z);
      if (z - f < 1e-9 || (f + 1.0) - z < 1e-9) fl = 1;
      int32_t c = (int32_t)f;
      key ^= (u32)c * P[a];
    }
    keys[i] = key;
    buckets[i] = nb_log2 >= 32 ? key : (key & ((1u << nb_log2) - 1u));
    if (flags) flags[i] = fl;
  }
}

// ---- Bucketing (Algorithm 1, distribute loop) ----
// Stable order of particle ids by bucket; rank = position of each id; each
// particle's bucket segment [seg_lo, seg_hi) in that order.
void or_bucket_sort(const u32* buckets, i64 np, int32_t* sorted_ids, int32_t* rank, int32_t* seg_lo,
                    int32_t* seg_hi) {
  std::vector<int32_t> ids(np);
  for (i64 i = 0; i < np; ++i) ids[i] = (int32_t)i;
  std::stable_sort(ids.begin(), ids.end(), [&](int32_t a, int32_t b) { return buckets[a] < buckets[b]; });
  for (i64 p = 0; p < np; ++p) { sorted_ids[p] = ids[p]; rank[ids[p]] = (int32_t)p; }
  i64 p = 0;
  while (p < np) {
    i64 q = p;
    while (q < np && buckets[ids[q]] == buckets[ids[p]]) ++q;
    for (i64 r = p; r < q; ++r) { seg_lo[ids[r]] = (int32_t)p; seg_hi[ids[r]] = (int32_t)q; }
    p = q;
  }
}

// ---- Neighbour list refinement (Algorithm 1 gather loop; Sec. III-C, lists
// kept across steps, K closest retained) ----
// Candidates of particle i: its previous list, and the bucket members at
// sorted positions [s, min(s + C, hi)), s = clamp(rank_i - C/2, lo,
// max(lo, hi - C)), where [lo, hi) is its bucket segment. Each candidate j != i
// gets d_ij = log(T_i^-1 T_j) and s_ij = sum_a W_aa d_a^2 (Eq. 7 and 8 as
// printed). The new list is i itself (s = 0) followed by the K-1 candidates of
// smallest (s_ij, j), sorted; k_ij = exp(-s_ij). Unused slots hold id -1.
// flags = 1 when the last kept and first dropped candidate are within tie_tol
// (relative) of each other.
void or_neighbor_merge(const float* poses, i64 np, const int32_t* old_ids, int K, int C,
                       const int32_t* sorted_ids, const int32_t* rank, const int32_t* seg_lo,
                       const int32_t* seg_hi, double sr, double st, double tie_tol, const int32_t* subset,
                       i64 n_subset, int32_t* ids, double* kk, double* dd, int32_t* flags, int nthreads) {
  // subset (optional): compute only these particles; output row r belongs to
  // particle subset[r].
  double W[6] = {sr, sr, sr, st, st, st};
  i64 n_out = subset ? n_subset : np;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 64)
#endif
  for (i64 row = 0; row < n_out; ++row) {
    i64 i = subset ? (i64)subset[row] : row;
    std::vector<int32_t> cand;
    if (old_ids)
      for (int a = 0; a < K; ++a) {
        int32_t j = old_ids[i * K + a];
        if (j >= 0 && j != i) cand.push_back(j);
      }
    i64 lo = seg_lo[i], hi = seg_hi[i], r = rank[i];
    i64 s = r - C / 2;
    i64 smax = std::max(lo, hi - (i64)C);
    if (s > smax) s = smax;
    if (s < lo) s = lo;
    i64 e = std::min(s + (i64)C, hi);
    for (i64 p = s; p < e; ++p) {
      int32_t j = sorted_ids[p];
      if (j != i) cand.push_back(j);
    }
    std::sort(cand.begin(), cand.end());
    cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
    Pose Ti = pose_from_f32(poses + 7 * i);
    struct E { double s; int32_t j; double d[6]; };
    std::vector<E> ev;
    ev.reserve(cand.size());
    for (int32_t j : cand) {
      E x;
      x.j = j;
      relative_log(Ti, pose_from_f32(poses + 7 * j), x.d);
      x.s = 0;
      for (int a = 0; a < 6; ++a) x.s += W[a] * x.d[a] * x.d[a];
      ev.push_back(x);
    }
    std::sort(ev.begin(), ev.end(), [](const E& a, const E& b) { return a.s < b.s || (a.s == b.s && a.j < b.j); });
    int keep = std::min<int>((int)ev.size(), K - 1);
    int fl = 0;
    if ((int)ev.size() > keep && keep > 0) {
      double a = ev[keep - 1].s, bb = ev[keep].s;
      if (bb - a <= tie_tol * std::max(bb, 1e-300)) fl = 1;
    }
    if (flags) flags[row] = fl;
    ids[row * K] = (int32_t)i;
    kk[row * K] = 1.0;
    for (int a = 0; a < 6; ++a) dd[(row * K) * 6 + a] = 0;
    for (int slot = 1; slot < K; ++slot) {
      i64 o = row * K + slot;
      if (slot - 1 < keep) {
        const E& x = ev[slot - 1];
        ids[o] = x.j;
        kk[o] = std::exp(-x.s);
        for (int a = 0; a < 6; ++a) dd[o * 6 + a] = x.d[a];
      } else {
        ids[o] = -1;
        kk[o] = 0;
        for (int a = 0; a < 6; ++a) dd[o * 6 + a] = 0;
      }
    }
  }
}

// ---- Scan-to-scan GICP odometry (Sec. III-B) ----
// Registers the current scan src (sensor frame at t) to the previous scan tgt
// (sensor frame at t-1): T = (R, t) maps src points into the tgt frame, so T
// estimates DeltaT_t = T_{t-1}^-1 T_t. Each iteration, for the current T:
//   * decisions in FP32: T's unit quaternion and translation rounded to
//     float, q_k = R32 mu_k + t32 (D1, D2); the correspondence of source point
//     k is the valid target point of smallest squared distance (D3), ties to
//     the smaller index, if that distance is <= r_corr^2;
//   * FP64 sums over the correspondences: e = mu^tgt - (R mu + t),
//     Omega = (Sigma^tgt + R Sigma^src R^T)^-1 (GICP planes),
//     J = R [ [mu]x , -I ] (right perturbation), H = sum J^T Omega J,
//     b = sum J^T Omega e (no truncation);
//   * delta = -(H + lambda diag H + eps I)^-1 b, T <- T exp(delta); stop when
//     max |delta_a| < tol or after max_iters iterations.
// Outputs the final T (4x4 row-major) and H of the last iteration (21 upper
// entries; Sigma^DeltaT = H^-1 is taken by the caller).
int or_gicp(const float* src, const double* src_n, const uint8_t* src_valid, i64 ns, const float* tgt,
            const double* tgt_n, const uint8_t* tgt_valid, i64 nt, const double* T0, double r_corr, double eps_cov,
            double lambda, double eps, int max_iters, double tol, double* T_out, double* H_out, int32_t* n_corr,
            int32_t* iters) {
  double R0[9];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) R0[3 * r + c] = T0[4 * r + c];
  Pose T;
  T.q = qnormalize(R_to_quat(R0));
  for (int a = 0; a < 3; ++a) T.t[a] = T0[4 * a + 3];
  const float r2 = (float)(r_corr * r_corr);
  double Hl[21] = {0};
  int cnt = 0, it = 0;
  std::vector<int> corr(ns);
  for (it = 0; it < max_iters; ++it) {
    // decisions on the FP32 rounding of T
    Quat qn = qnormalize(T.q);
    float P32[7] = {(float)qn.x, (float)qn.y, (float)qn.z, (float)qn.w, (float)T.t[0], (float)T.t[1], (float)T.t[2]};
    float R32[9];
    R32_of(P32, R32);
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (i64 k = 0; k < ns; ++k) {
      corr[k] = -1;
      if (src_valid && !src_valid[k]) continue;
      float q32[3];
      transform32(R32, P32 + 4, src + 3 * k, q32);
      float best = INFINITY;
      int bj = -1;
      for (i64 j = 0; j < nt; ++j) {
        if (tgt_valid && !tgt_valid[j]) continue;
        float d2 = dist2_32(q32, tgt + 3 * j);
        if (d2 < best) { best = d2; bj = (int)j; }
      }
      if (bj >= 0 && best <= r2) corr[k] = bj;
    }
    // FP64 sums
    double R[9];
    quat_to_R(qn, R);
    double b[6] = {0};
    for (int a = 0; a < 21; ++a) Hl[a] = 0;
    cnt = 0;
    for (i64 k = 0; k < ns; ++k) {
      int m = corr[k];
      if (m < 0) continue;
      double mus[3] = {src[3 * k], src[3 * k + 1], src[3 * k + 2]};
      double qk[3];
      matvec3(R, mus, qk);
      double e[3];
      for (int a = 0; a < 3; ++a) e[a] = (double)tgt[3 * m + a] - (qk[a] + T.t[a]);
      double SM[9], SS[9], RS[9], RSRt[9], Rt[9], C[9], Om[9];
      gicp_cov(tgt_n + 3 * m, eps_cov, SM);
      gicp_cov(src_n + 3 * k, eps_cov, SS);
      for (int r = 0; r < 3; ++r) for (int c = 0; c < 3; ++c) Rt[3 * r + c] = R[3 * c + r];
      matmul3(R, SS, RS);
      matmul3(RS, Rt, RSRt);
      for (int a = 0; a < 9; ++a) C[a] = SM[a] + RSRt[a];
      if (!inv3(C, Om)) continue;
      cnt++;
      double Oe[3];
      matvec3(Om, e, Oe);
      double S[9], J0[9], J[3][6];
      skew(mus, S);
      matmul3(R, S, J0);
      for (int r = 0; r < 3; ++r)
        for (int c2 = 0; c2 < 3; ++c2) { J[r][c2] = J0[3 * r + c2]; J[r][3 + c2] = -R[3 * r + c2]; }
      for (int a = 0; a < 6; ++a) {
        for (int bb = a; bb < 6; ++bb) {
          double sacc = 0;
          for (int r = 0; r < 3; ++r)
            sacc += J[r][a] * (Om[3 * r] * J[0][bb] + Om[3 * r + 1] * J[1][bb] + Om[3 * r + 2] * J[2][bb]);
          Hl[H_IDX[a][bb]] += sacc;
        }
        double sacc = 0;
        for (int r = 0; r < 3; ++r) sacc += J[r][a] * Oe[r];
        b[a] += sacc;
      }
    }
    // damped Gauss-Newton step
    double A[36], d[6];
    for (int a = 0; a < 6; ++a)
      for (int c = 0; c < 6; ++c) A[6 * a + c] = Hl[H_IDX[a][c]];
    for (int a = 0; a < 6; ++a) A[7 * a] += lambda * A[7 * a] + eps;
    // Gaussian elimination with partial pivoting on the 6x6 system A d = -b
    double M[6][7];
    for (int a = 0; a < 6; ++a) {
      for (int c = 0; c < 6; ++c) M[a][c] = A[6 * a + c];
      M[a][6] = -b[a];
    }
    bool ok = cnt >= 6;
    for (int c = 0; c < 6 && ok; ++c) {
      int piv = c;
      for (int r = c + 1; r < 6; ++r)
        if (std::fabs(M[r][c]) > std::fabs(M[piv][c])) piv = r;
      if (!(std::fabs(M[piv][c]) > 0)) { ok = false; break; }
      if (piv != c) for (int k = 0; k < 7; ++k) std::swap(M[c][k], M[piv][k]);
      for (int r = c + 1; r < 6; ++r) {
        double f = M[r][c] / M[c][c];
        for (int k = c; k < 7; ++k) M[r][k] -= f * M[c][k];
      }
    }
    if (!ok) break;
    for (int r = 5; r >= 0; --r) {
      double v = M[r][6];
      for (int k = r + 1; k < 6; ++k) v -= M[r][k] * d[k];
      d[r] = v / M[r][r];
    }
    T = compose(T, se3_exp(d));
    T.q = qnormalize(T.q);
    double mx = 0;
    for (int a = 0; a < 6; ++a) mx = std::max(mx, std::fabs(d[a]));
    if (mx < tol) { ++it; break; }
  }
  double R[9];
  quat_to_R(qnormalize(T.q), R);
  for (int r = 0; r < 3; ++r) {
    for (int c = 0; c < 3; ++c) T_out[4 * r + c] = R[3 * r + c];
    T_out[4 * r + 3] = T.t[r];
  }
  T_out[12] = T_out[13] = T_out[14] = 0.0;
  T_out[15] = 1.0;
  if (H_out) for (int a = 0; a < 21; ++a) H_out[a] = Hl[a];
  if (n_corr) *n_corr = cnt;
  if (iters) *iters = it;
  return 0;
}

// ---- SVGD update (Sec. III-C Eq. 5 and 6) ----
// phi_i = sum_j (k_ij psi_j + grad_{T_j} k(T_i, T_j)) / sum_j k_ij over the
// list of i, with grad_{T_j} k = -2 k_ij W^K d_ij (d_ij in T_i's tangent
// space, first order in the perturbation of T_j); T_i <- T_i exp(phi_i).
// pinv (optional, np x 36 row-major): the repulsive sum of particle i is
// multiplied by pinv_i (a Stein variational Newton reading that scales the
// repulsion like the Gauss-Newton steps psi_j; not the paper's printed form).
void or_svgd(const float* poses, i64 np, const int32_t* ids, const double* kk, const double* dd, int K,
             const double* psi, double sr, double st, const double* pinv, double* phi, double* poses_out) {
  double W[6] = {sr, sr, sr, st, st, st};
  for (i64 i = 0; i < np; ++i) {
    double att[6] = {0}, rep[6] = {0}, den = 0;
    for (int slot = 0; slot < K; ++slot) {
      i64 o = i * K + slot;
      int32_t j = ids[o];
      if (j < 0) continue;
      double k = kk[o];
      den += k;
      for (int a = 0; a < 6; ++a) {
        att[a] += k * psi[6 * j + a];
        rep[a] += -2.0 * k * W[a] * dd[o * 6 + a];
      }
    }
    double num[6];
    for (int a = 0; a < 6; ++a) {
      double r = rep[a];
      if (pinv) {
        r = 0;
        for (int c = 0; c < 6; ++c) r += pinv[36 * i + 6 * a + c] * rep[c];
      }
      num[a] = att[a] + r;
    }
    double ph[6];
    for (int a = 0; a < 6; ++a) ph[a] = den > 0 ? num[a] / den : 0.0;
    if (phi) for (int a = 0; a < 6; ++a) phi[6 * i + a] = ph[a];
    Pose T = pose_from_f32(poses + 7 * i);
    Pose N = compose(T, se3_exp(ph));
    N.q = qnormalize(N.q);
    poses_out[7 * i] = N.q.x; poses_out[7 * i + 1] = N.q.y; poses_out[7 * i + 2] = N.q.z; poses_out[7 * i + 3] = N.q.w;
    for (int a = 0; a < 3; ++a) poses_out[7 * i + 4 + a] = N.t[a];
  }
}

// ---- Posterior propagation (Sec. III-D, Eq. 11) ----
// p(x_i | P) proportional to p(x_i) p(P | x_i), in the log domain:
// l_i = logprior_i + loglik_i, p_i = exp(l_i - max l) / sum (FP64). Then
// `iters` Jacobi sweeps p'_i = sum_j k_ij p_j / sum_j k_ij over the list of i,
// and a final renormalisation. best = argmax p' (smallest index on ties).
void or_posterior(const double* logprior, const double* loglik, i64 np, const int32_t* ids, const double* kk,
                  int K, int iters, double floor_nats, double* p_init, double* p_out, i64* best) {
  std::vector<double> l(np), p(np), q(np);
  double mx = -INFINITY;
  for (i64 i = 0; i < np; ++i) {
    l[i] = (logprior ? logprior[i] : 0.0) + (loglik ? loglik[i] : 0.0);
    if (l[i] > mx) mx = l[i];
  }
  // the initial posterior relative to its largest value, exp(l - max l), is
  // kept at or above exp(-floor_nats) (floor_nats = 0: no floor): no particle's
  // posterior, and so no particle's prior at the next step, is an exact zero
  const double lo = floor_nats > 0 ? -floor_nats : -INFINITY;
  double sum = 0;
  for (i64 i = 0; i < np; ++i) { p[i] = std::exp(std::max(l[i] - mx, lo)); sum += p[i]; }
  for (i64 i = 0; i < np; ++i) p[i] /= sum;
  if (p_init) for (i64 i = 0; i < np; ++i) p_init[i] = p[i];
  for (int it = 0; it < iters; ++it) {
    for (i64 i = 0; i < np; ++i) {
      double num = 0, den = 0;
      for (int slot = 0; slot < K; ++slot) {
        int32_t j = ids[i * K + slot];
        if (j < 0) continue;
        num += kk[i * K + slot] * p[j];
        den += kk[i * K + slot];
      }
      q[i] = den > 0 ? num / den : p[i];
    }
    std::swap(p, q);
  }
  sum = 0;
  for (i64 i = 0; i < np; ++i) sum += p[i];
  i64 bi = 0;
  for (i64 i = 0; i < np; ++i) {
    p_out[i] = p[i] / sum;
    if (p_out[i] > p_out[bi]) bi = i;
  }
  if (best) *best = bi;
}

// ---- Prediction (Sec. III-B Eq. 1) ----
// T_i <- T_i dT exp(delta_i), delta_i = L n_i, L the lower Cholesky factor of
// Sigma^dT (columns with a non-positive pivot are zero), n_i six standard
// normals: Box-Muller on the 32-bit uniforms of counters (i, 0, step,
// STREAM_PREDICT) (pairs (0,1), (2,3)) and (i, 1, step, STREAM_PREDICT)
// (pair (0,1)).
void or_cholesky6(const double S[36], double L[36]) {
  for (int a = 0; a < 36; ++a) L[a] = 0;
  for (int j = 0; j < 6; ++j) {
    double d = S[6 * j + j];
    for (int k = 0; k < j; ++k) d -= L[6 * j + k] * L[6 * j + k];
    if (!(d > 1e-300)) continue;
    double s = std::sqrt(d);
    L[6 * j + j] = s;
    for (int r = j + 1; r < 6; ++r) {
      double v = S[6 * r + j];
      for (int k = 0; k < j; ++k) v -= L[6 * r + k] * L[6 * j + k];
      L[6 * r + j] = v / s;
    }
  }
}

void or_predict_noise(i64 i, u64 seed, u64 step, double n[6]) {
  u32 key[2] = {(u32)seed, (u32)(seed >> 32)};
  u32 c0[4] = {(u32)i, 0u, (u32)step, STREAM_PREDICT}, c1[4] = {(u32)i, 1u, (u32)step, STREAM_PREDICT};
  u32 o0[4], o1[4];
  philox(c0, key, o0);
  philox(c1, key, o1);
  u32 pairs[3][2] = {{o0[0], o0[1]}, {o0[2], o0[3]}, {o1[0], o1[1]}};
  const double two_pi = 6.283185307179586476925286766559;
  for (int p = 0; p < 3; ++p) {
    double r = std::sqrt(-2.0 * std::log(uniform32(pairs[p][0])));
    double th = two_pi * uniform32(pairs[p][1]);
    n[2 * p] = r * std::cos(th);
    n[2 * p + 1] = r * std::sin(th);
  }
}

void or_predict(const float* poses, i64 np, const double odom_T[16], const double odom_cov[36], u64 seed,
                u64 step, double* poses_out, double* delta_out) {
  double Rd[9] = {odom_T[0], odom_T[1], odom_T[2], odom_T[4], odom_T[5], odom_T[6], odom_T[8], odom_T[9], odom_T[10]};
  Pose D;
  D.q = R_to_quat(Rd);
  D.t[0] = odom_T[3]; D.t[1] = odom_T[7]; D.t[2] = odom_T[11];
  double L[36];
  or_cholesky6(odom_cov, L);
  for (i64 i = 0; i < np; ++i) {
    double n[6], d[6];
    or_predict_noise(i, seed, step, n);
    for (int r = 0; r < 6; ++r) {
      d[r] = 0;
      for (int c = 0; c <= r; ++c) d[r] += L[6 * r + c] * n[c];
    }
    if (delta_out) for (int r = 0; r < 6; ++r) delta_out[6 * i + r] = d[r];
    Pose T = pose_from_f32(poses + 7 * i);
    Pose N = compose(compose(T, D), se3_exp(d));
    N.q = qnormalize(N.q);
    poses_out[7 * i] = N.q.x; poses_out[7 * i + 1] = N.q.y; poses_out[7 * i + 2] = N.q.z; poses_out[7 * i + 3] = N.q.w;
    for (int a = 0; a < 3; ++a) poses_out[7 * i + 4 + a] = N.t[a];
  }
}

// ---- Uniform initialisation (Sec. IV-A: particles uniform over the map box)
// Six 32-bit uniforms per particle from counters (i, 0, 0, STREAM_INIT) and
// (i, 1, 0, STREAM_INIT) (first two words): x, y, z, roll, pitch, yaw uniform
// in [lo, hi], R = Rz(yaw) Ry(pitch) Rx(roll). When every angle range spans at
// least 2 pi the rotation is instead uniform on SO(3) (Shoemake, from the
// three angle uniforms u3, u4, u5).
void or_init_uniform(i64 np, const double lo[6], const double hi[6], u64 seed, double* poses_out) {
  u32 key[2] = {(u32)seed, (u32)(seed >> 32)};
  const double two_pi = 6.283185307179586476925286766559;
  bool full = true;
  for (int a = 3; a < 6; ++a) if (hi[a] - lo[a] < two_pi) full = false;
  for (i64 i = 0; i < np; ++i) {
    u32 c0[4] = {(u32)i, 0u, 0u, STREAM_INIT}, c1[4] = {(u32)i, 1u, 0u, STREAM_INIT};
    u32 o0[4], o1[4];
    philox(c0, key, o0);
    philox(c1, key, o1);
    double u[6] = {uniform32(o0[0]), uniform32(o0[1]), uniform32(o0[2]), uniform32(o0[3]),
                   uniform32(o1[0]), uniform32(o1[1])};
    double v[6];
    for (int a = 0; a < 6; ++a) v[a] = lo[a] + u[a] * (hi[a] - lo[a]);
    Quat q;
    if (full) {
      double a = std::sqrt(1.0 - u[3]), bq = std::sqrt(u[3]);
      q = Quat{a * std::sin(two_pi * u[4]), a * std::cos(two_pi * u[4]), bq * std::sin(two_pi * u[5]),
               bq * std::cos(two_pi * u[5])};
    } else {
      double cr = std::cos(0.5 * v[3]), sr = std::sin(0.5 * v[3]);
      double cp = std::cos(0.5 * v[4]), sp = std::sin(0.5 * v[4]);
      double cy = std::cos(0.5 * v[5]), sy = std::sin(0.5 * v[5]);
      Quat qx{sr, 0, 0, cr}, qy{0, sp, 0, cp}, qz{0, 0, sy, cy};
      q = qmul(qz, qmul(qy, qx));
    }
    q = qnormalize(q);
    poses_out[7 * i] = q.x; poses_out[7 * i + 1] = q.y; poses_out[7 * i + 2] = q.z; poses_out[7 * i + 3] = q.w;
    for (int a = 0; a < 3; ++a) poses_out[7 * i + 4 + a] = v[a];
  }
}

}  // extern "C"
