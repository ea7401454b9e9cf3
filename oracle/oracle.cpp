// FP64 CPU oracle of the batched compliant-tree step.
//
// TEST INFRASTRUCTURE ONLY. Nothing in the product path may link, load or call this file:
// only the tests, the smoke check and the benchmark's CPU-baseline leg use it. It shares no
// code, header, table or helper with the CUDA path; the two meet only through the seeded
// inputs of paper_2607_06337_b300/inputs.py.
//
// It is written for a reader checking it against the paper, not for speed:
//   * kinematics: joint rest transform T = (0,0,l_parent) * q_rel (Sec. IV, Eq. 3), each
//     compliant joint as two bending hinges (Cardan x then y') of a twist-locked D6 (Sec. IV-A);
//   * mass matrix by its definition M = sum_b J_b^T diag(m_b, I_b) J_b over body Jacobians
//     (no composite-inertia recursion);
//   * bias forces by the virtual-work projection c = sum_b J_b^T (Newton-Euler wrench of b)
//     with classical (not spatial) accelerations, minus the generalised apple reactions;
//   * stiffness k and rupture moment from the descriptor (Sec. IV-A Eq. 4, Sec. IV-B Eq. 5),
//     restoring torque -k theta - kd omega with implicit damping (and, by flag, implicit
//     springs: "exact implicit position actuators", Sec. IV-A);
//   * H = M + diag(armature) + dt diag(kd') + alpha dt^2 diag(k') (+ dt^2 k_s J_h^T J_h per
//     attached apple when the tether reaction is taken implicitly), solved densely (LDL^T)
//     for small trees and by the tree-sparse LTDL factorisation for large ones;
//   * tether, reaction, clamp and detachment (Sec. IV-C, Eqs. 6-7), rupture with hysteresis
//     (Sec. IV-B, Eq. 5), semi-implicit update;
//   * velocity-proportional damping of the bodies, force -c_v m v and torque -c_omega I omega
//     at the centre of mass (Sec. IV-A), with the linear part reduced on a snapped sub-tree
//     (Sec. IV-B), taken explicitly at the step's start velocities;
//   * the three rails on the applied force of an apple (App. B: impulse cap, power fade, speed
//     brake), at the step's start velocity.
// Every function is templated on the scalar so the same code runs in double and in
// std::complex<double> (complex-step derivatives for the adjoint checks).
//
// Parity pins live in tests/test_oracle_*.py (closed forms, brute force, invariants).

#include <algorithm>
#include <atomic>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <thread>
#include <vector>

namespace {

using cplx = std::complex<double>;
// single-precision complex step: the same derivative with every operation rounded to FP32
// (the rounding floor of an FP32 evaluation of a gradient, for the adjoint's tolerance)
using cplxf = std::complex<float>;

inline double re(double x) { return x; }
inline double re(const cplx& x) { return x.real(); }
inline double re(const cplxf& x) { return x.real(); }

// Reverse-mode scalar: the oracle's own adjoint. Every operation on an RV appends one node
// to the current thread's tape (its value's local partial derivatives with respect to at most
// two operands); one backward pass over the tape then gives the derivative of a final value
// with respect to every leaf. Comparisons use the value, so event masks stay as in the plain
// run, exactly like the complex-step and the GPU adjoint.
struct Tape {
  std::vector<int32_t> pa, pb;  // operand nodes (-1: a constant)
  std::vector<double> ga, gb;   // d(node)/d(operand)
  int32_t push(int32_t a, double da, int32_t b, double db) {
    pa.push_back(a); ga.push_back(da); pb.push_back(b); gb.push_back(db);
    return (int32_t)pa.size() - 1;
  }
};
Tape*& tape_slot() {
  static thread_local Tape* t = nullptr;
  return t;
}
struct RV {
  double v = 0.0;
  int32_t id = -1;  // -1: a constant (no derivative)
  RV() = default;
  RV(double x) : v(x), id(-1) {}
  static RV node(double v, int32_t a, double da, int32_t b, double db) {
    RV r;
    r.v = v;
    if (a >= 0 || b >= 0) r.id = tape_slot()->push(a, da, b, db);
    return r;
  }
  static RV leaf(double v) {
    RV r;
    r.v = v;
    r.id = tape_slot()->push(-1, 0.0, -1, 0.0);
    return r;
  }
};
inline double re(const RV& x) { return x.v; }
inline RV operator+(const RV& x, const RV& y) { return RV::node(x.v + y.v, x.id, 1.0, y.id, 1.0); }
inline RV operator-(const RV& x, const RV& y) { return RV::node(x.v - y.v, x.id, 1.0, y.id, -1.0); }
inline RV operator*(const RV& x, const RV& y) { return RV::node(x.v * y.v, x.id, y.v, y.id, x.v); }
inline RV operator/(const RV& x, const RV& y) {
  const double q = x.v / y.v;
  return RV::node(q, x.id, 1.0 / y.v, y.id, -q / y.v);
}
inline RV operator-(const RV& x) { return RV::node(-x.v, x.id, -1.0, -1, 0.0); }
inline RV& operator+=(RV& x, const RV& y) { return x = x + y; }
inline RV& operator-=(RV& x, const RV& y) { return x = x - y; }
inline RV& operator*=(RV& x, const RV& y) { return x = x * y; }
inline RV& operator/=(RV& x, const RV& y) { return x = x / y; }
// the std overloads stay visible beside the RV ones for double and std::complex<double>
using std::cos;
using std::sin;
using std::sqrt;
inline RV sin(const RV& x) { return RV::node(std::sin(x.v), x.id, std::cos(x.v), -1, 0.0); }
inline RV cos(const RV& x) { return RV::node(std::cos(x.v), x.id, -std::sin(x.v), -1, 0.0); }
inline RV sqrt(const RV& x) {
  const double r = std::sqrt(x.v);
  return RV::node(r, x.id, 0.5 / r, -1, 0.0);
}

// d(out)/d(node) for every node of the tape (nodes whose adjoint is zero are skipped, so an
// unused infinite partial, e.g. of sqrt at 0, cannot turn into 0 * inf).
std::vector<double> tape_adjoints(const Tape& t, int32_t out) {
  std::vector<double> adj(t.pa.size(), 0.0);
  if (out < 0) return adj;
  adj[out] = 1.0;
  for (int32_t i = out; i >= 0; --i) {
    const double a = adj[i];
    if (a == 0.0) continue;
    if (t.pa[i] >= 0) adj[t.pa[i]] += a * t.ga[i];
    if (t.pb[i] >= 0) adj[t.pb[i]] += a * t.gb[i];
  }
  return adj;
}

template <class T> struct V3 {
  T x, y, z;
};
template <class T> inline V3<T> v3(T a, T b, T c) { return {a, b, c}; }
template <class T> inline V3<T> operator+(const V3<T>& a, const V3<T>& b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
template <class T> inline V3<T> operator-(const V3<T>& a, const V3<T>& b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
template <class T> inline V3<T> operator*(const T& s, const V3<T>& a) { return {s * a.x, s * a.y, s * a.z}; }
template <class T> inline T dot(const V3<T>& a, const V3<T>& b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <class T> inline V3<T> cross(const V3<T>& a, const V3<T>& b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}

// 3x3 matrix, row-major.
template <class T> struct M3 {
  T a[9];
};
template <class T> inline M3<T> mmul(const M3<T>& A, const M3<T>& B) {
  M3<T> C;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      T s = T(0);
      for (int k = 0; k < 3; ++k) s += A.a[3 * i + k] * B.a[3 * k + j];
      C.a[3 * i + j] = s;
    }
  return C;
}
template <class T> inline V3<T> mvec(const M3<T>& A, const V3<T>& v) {
  return {A.a[0] * v.x + A.a[1] * v.y + A.a[2] * v.z, A.a[3] * v.x + A.a[4] * v.y + A.a[5] * v.z,
          A.a[6] * v.x + A.a[7] * v.y + A.a[8] * v.z};
}
template <class T> inline V3<T> col(const M3<T>& A, int j) { return {A.a[j], A.a[3 + j], A.a[6 + j]}; }
template <class T> inline M3<T> eye3() {
  M3<T> I;
  for (int i = 0; i < 9; ++i) I.a[i] = T(0);
  I.a[0] = I.a[4] = I.a[8] = T(1);
  return I;
}
template <class T> inline M3<T> rot_x(T t) {
  T c = cos(t), s = sin(t);
  M3<T> R = eye3<T>();
  R.a[4] = c; R.a[5] = -s; R.a[7] = s; R.a[8] = c;
  return R;
}
template <class T> inline M3<T> rot_y(T t) {
  T c = cos(t), s = sin(t);
  M3<T> R = eye3<T>();
  R.a[0] = c; R.a[2] = s; R.a[6] = -s; R.a[8] = c;
  return R;
}
// unit quaternion (w,x,y,z) -> rotation matrix
template <class T> inline M3<T> quat_mat(const double* q) {
  double w = q[0], x = q[1], y = q[2], z = q[3];
  double n = std::sqrt(w * w + x * x + y * y + z * z);
  w /= n; x /= n; y /= n; z /= n;
  M3<T> R;
  R.a[0] = T(1 - 2 * (y * y + z * z)); R.a[1] = T(2 * (x * y - w * z)); R.a[2] = T(2 * (x * z + w * y));
  R.a[3] = T(2 * (x * y + w * z)); R.a[4] = T(1 - 2 * (x * x + z * z)); R.a[5] = T(2 * (y * z - w * x));
  R.a[6] = T(2 * (x * z - w * y)); R.a[7] = T(2 * (y * z + w * x)); R.a[8] = T(1 - 2 * (x * x + y * y));
  return R;
}
template <class T> inline V3<T> dv(const double* p) { return {T(p[0]), T(p[1]), T(p[2])}; }

}  // namespace

// ------------------------------------------------------------------------------------------
// C ABI structures (mirrored by ctypes in oracle/__init__.py).
// ------------------------------------------------------------------------------------------
extern "C" {

typedef struct {
  int32_t n_worlds;
  const int32_t *body_off, *apple_off, *tip_off;
  const int32_t *parent, *ndof;
  const double *jpos, *qrel, *com, *mass, *inertia, *k, *kd, *armature, *m_max;
  const int32_t* apple_body;
  const double *hang_local, *apple_mass, *k_s, *c_s, *f_detach;
  const int32_t* tip_body;
  const double *tip_local, *gravity;
} OForest;

typedef struct {
  double dt;
  int32_t alpha_implicit_spring, tether_implicit, n_break, n_pull, n_tension;
  double gamma_tension, clamp_factor;
  int32_t dense_limit;  // solve densely when n_v <= dense_limit, else by tree LTDL
  double break_ramp_s;      // post-break friction surrogate ramps over this time (s)
  double break_ramp_factor; // ... from kd to this multiple of kd
  double lin_damping;       // c_v (1/s): force -c_v m v at each body's centre of mass
  double ang_damping;       // c_omega (1/s): torque -c_omega I omega
  double snapped_lin_damping;  // factor on c_v for a body on a snapped sub-tree
  double rail_speed;        // v_lim (m/s) of the applied-force rails, 0: rails off
  double rail_fade_speed;   // v_fade (m/s), 0 <= v_fade < v_lim
  double rail_brake;        // c_b (1/s) of the speed brake
} OFlags;

typedef struct {
  double *q, *qd;                         // [n_v total]
  double *ax, *av;                        // [n_apples total][3]
  int32_t *broken, *bcnt, *break_step;    // [n_bodies total]
  int32_t *detached, *pcnt, *tcnt, *detach_step;  // [n_apples total]
  int32_t* status;                        // [n_worlds] bit 0: non-finite state
} OState;

typedef struct {
  const double* force;  // [n_apples total][3]
  const int32_t *start, *end;
} OPulls;

typedef struct {
  double* tips;         // [n_steps][n_tips total][3] tip positions after each step, or NULL
  double* q;            // [n_steps][n_v total] joint positions after each step, or NULL
  int32_t* near;        // [near_cap][4] (world, kind 0 break/1 pull/2 tension, index, step)
  double* near_margin;  // [near_cap]
  int32_t near_cap;
  int32_t* near_count;  // number written (may exceed cap: entries past cap are dropped)
  double near_eps;      // log every test whose relative margin is below this
} ORecord;

}  // extern "C"

namespace {

// One world's view into the packed forest.
struct World {
  int nb, na, nt, nv;
  const int32_t *parent, *ndof;
  const double *jpos, *qrel, *com, *mass, *inertia, *k, *kd, *arm, *m_max;
  const int32_t* abody;
  const double *hang, *am, *ks, *cs, *fdet;
  const int32_t* tbody;
  const double* tlocal;
  const double* g;
  std::vector<int> dof0;       // first DOF of each body
  std::vector<int> dof_body;   // body of each DOF
  std::vector<int> dof_parent; // DOF-tree parent (lambda), -1 at the top
  std::vector<std::vector<int>> chain;  // DOFs of the body and all its ancestors
};

World make_world(const OForest* f, int w) {
  World W;
  int b0 = f->body_off[w], b1 = f->body_off[w + 1];
  int a0 = f->apple_off[w], a1 = f->apple_off[w + 1];
  int t0 = f->tip_off[w], t1 = f->tip_off[w + 1];
  W.nb = b1 - b0; W.na = a1 - a0; W.nt = t1 - t0;
  W.parent = f->parent + b0; W.ndof = f->ndof + b0;
  W.jpos = f->jpos + 3 * b0; W.qrel = f->qrel + 4 * b0; W.com = f->com + 3 * b0;
  W.mass = f->mass + b0; W.inertia = f->inertia + 3 * b0; W.k = f->k + b0; W.kd = f->kd + b0;
  W.arm = f->armature + b0; W.m_max = f->m_max + b0;
  W.abody = f->apple_body + a0; W.hang = f->hang_local + 3 * a0;
  W.am = f->apple_mass + a0; W.ks = f->k_s + a0; W.cs = f->c_s + a0; W.fdet = f->f_detach + a0;
  W.tbody = f->tip_body + t0; W.tlocal = f->tip_local + 3 * t0;
  W.g = f->gravity + 3 * w;
  W.dof0.resize(W.nb);
  int n = 0;
  for (int b = 0; b < W.nb; ++b) { W.dof0[b] = n; n += W.ndof[b]; }
  W.nv = n;
  W.dof_body.resize(n);
  W.dof_parent.resize(n);
  W.chain.resize(W.nb);
  for (int b = 0; b < W.nb; ++b) {
    int p = W.parent[b];
    if (p >= 0) W.chain[b] = W.chain[p];
    for (int j = 0; j < W.ndof[b]; ++j) {
      int i = W.dof0[b] + j;
      W.dof_body[i] = b;
      W.dof_parent[i] = W.chain[b].empty() ? -1 : W.chain[b].back();
      W.chain[b].push_back(i);
    }
  }
  return W;
}

int dof_offset(const OForest* f, int w) {
  int n = 0;
  for (int b = 0; b < f->body_off[w]; ++b) n += f->ndof[b];
  return n;
}

// Kinematics of one configuration.
template <class T> struct Kin {
  std::vector<M3<T>> R;       // body rotation (world)
  std::vector<V3<T>> x;       // joint origin (world)
  std::vector<V3<T>> c;       // centre of mass (world)
  std::vector<V3<T>> e;       // DOF axes (world), through x of the DOF's body
  std::vector<V3<T>> w;       // body angular velocity
  std::vector<V3<T>> vx;      // velocity of the joint origin
  std::vector<V3<T>> al;      // angular acceleration at qdd = 0
  std::vector<V3<T>> ax;      // acceleration of the joint origin at qdd = 0
};

// Forward kinematics: R_b = R_p Rot(q_rel) Rx(theta_0) Ry(theta_1), x_b = x_p + R_p jpos_b
// (Sec. IV, Eq. 3; Sec. IV-A two bending DOFs), then velocities and the velocity-product
// accelerations of each body with joint accelerations set to zero (classical kinematics).
template <class T>
void kinematics(const World& W, const T* q, const T* qd, Kin<T>& K) {
  K.R.resize(W.nb); K.x.resize(W.nb); K.c.resize(W.nb); K.e.resize(W.nv);
  K.w.resize(W.nb); K.vx.resize(W.nb); K.al.resize(W.nb); K.ax.resize(W.nb);
  const V3<T> zero = {T(0), T(0), T(0)};
  for (int b = 0; b < W.nb; ++b) {
    int p = W.parent[b];
    M3<T> Rp = p >= 0 ? K.R[p] : eye3<T>();
    V3<T> xp = p >= 0 ? K.x[p] : zero;
    V3<T> wp = p >= 0 ? K.w[p] : zero;
    V3<T> vp = p >= 0 ? K.vx[p] : zero;
    V3<T> alp = p >= 0 ? K.al[p] : zero;
    V3<T> axp = p >= 0 ? K.ax[p] : zero;
    M3<T> Rj = mmul(Rp, quat_mat<T>(W.qrel + 4 * b));
    V3<T> xb = xp + mvec(Rp, dv<T>(W.jpos + 3 * b));
    V3<T> d = xb - xp;
    // the joint origin is a point fixed in the parent
    K.vx[b] = vp + cross(wp, d);
    K.ax[b] = axp + cross(alp, d) + cross(wp, cross(wp, d));
    M3<T> Rb = Rj;
    V3<T> wb = wp, alb = alp;
    int i0 = W.dof0[b];
    for (int j = 0; j < W.ndof[b]; ++j) {
      V3<T> ej = col(Rb, j);            // x of the joint frame, then y' after the first turn
      K.e[i0 + j] = ej;
      alb = alb + qd[i0 + j] * cross(wb, ej);  // d/dt of the moving axis times its rate
      wb = wb + qd[i0 + j] * ej;
      Rb = mmul(Rb, j == 0 ? rot_x(q[i0 + j]) : rot_y(q[i0 + j]));
    }
    K.R[b] = Rb; K.x[b] = xb; K.w[b] = wb; K.al[b] = alb;
    K.c[b] = xb + mvec(Rb, dv<T>(W.com + 3 * b));
  }
}

template <class T> inline M3<T> world_inertia(const World& W, const Kin<T>& K, int b) {
  // R diag(I) R^T about the centre of mass
  M3<T> D = eye3<T>();
  D.a[0] = T(W.inertia[3 * b]); D.a[4] = T(W.inertia[3 * b + 1]); D.a[8] = T(W.inertia[3 * b + 2]);
  M3<T> Rt;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) Rt.a[3 * i + j] = K.R[b].a[3 * j + i];
  return mmul(mmul(K.R[b], D), Rt);
}

// Linear-velocity Jacobian column of a world point p fixed in the subtree of DOF i.
template <class T> inline V3<T> jac_point(const World& W, const Kin<T>& K, int i, const V3<T>& p) {
  return cross(K.e[i], p - K.x[W.dof_body[i]]);
}

// Per-step apple forces on the tree (Sec. IV-C). An attached apple's state is its stem
// elongation u = x - x_hang (so du/dt = v - v_hang); the stem force on it is
// f_s = -k_s u (Eq. 6); the spur receives f_react = -(f_s - m g z) = -(f_s + m g_vec),
// clamped in norm (Eq. 7). Reading of the time integration: the tether is stepped by backward
// Euler in its elongation for the apple and the tree together. The apple's new velocity is
// v' = a + beta v_hang' with a = (m v + dt (f_ext + m g + f_s)) / D, beta = dt^2 k_s / D,
// D = m + dt c_s + dt^2 k_s; eliminating it leaves the tree with the force
// f_react + dt k_s a - dt kappa v_hang at the hang point and dt^2 kappa J_h^T J_h in H,
// kappa = k_s (1 - beta). Reading of the clamp (Eq. 7, "clamped to a maximum"): when
// |f_react| > F_clamp the coupled reaction, force and stiffness alike, is scaled by
// F_clamp / |f_react| (continuous at the threshold). In the explicit mode the plain clamped
// f_react is applied and v' = a. Detached apples, and apples on a snapped sub-tree (whose
// applied forces are disabled, App. B), give nothing.
template <class T> struct AppleLoads {
  std::vector<V3<T>> hang;     // world hang point
  std::vector<V3<T>> vhang;    // its velocity at the start of the step
  std::vector<V3<T>> fapp;     // force applied to the tree at the hang point
  std::vector<V3<T>> a;        // apple velocity with the hang point frozen
  std::vector<T> beta;         // coupling of the new apple velocity to the new hang velocity
  std::vector<T> kappa;        // coupling stiffness added to H (0: none)
  std::vector<T> tension, pull;
};

// A body is on a snapped sub-tree when its own joint or any joint above it is broken.
std::vector<int> snapped_bodies(const World& W, const int32_t* broken) {
  std::vector<int> s(W.nb, 0);
  for (int b = 0; b < W.nb; ++b) s[b] = (broken && broken[b]) || (W.parent[b] >= 0 && s[W.parent[b]]);
  return s;
}

// The three rails of App. B on the applied force f of a body of mass m and velocity v (this
// step's start):
//   (1) impulse cap: the velocity f alone adds in one step, dt |f| / m, is at most v_lim;
//   (2) power fade: the component of f along v, when it pushes along v, fades linearly from
//       full at |v| = v_fade to none at |v| = v_lim;
//   (3) speed brake: above v_lim, -c_b m (|v| - v_lim) v / |v| is added.
// Rails off (v_lim = 0) or no applied force: f unchanged. At rest, below the cap, nothing
// changes ("none of which affects static loading").
template <class T> V3<T> rails(const OFlags& fl, T m, V3<T> v, V3<T> f) {
  if (!(fl.rail_speed > 0)) return f;
  T fn = sqrt(dot(f, f));
  if (re(fn) == 0.0) return f;
  const double vl = fl.rail_speed, vf = fl.rail_fade_speed;
  T cap = m * T(vl / fl.dt);
  if (re(fn) > re(cap)) f = (cap / fn) * f;
  T s = sqrt(dot(v, v));
  if (re(s) > vf) {
    V3<T> vh = (T(1) / s) * v;
    T p = dot(f, vh);
    if (re(p) > 0) {
      T phi = re(s) >= vl ? T(0) : (T(vl) - s) / T(vl - vf);
      f = f - ((T(1) - phi) * p) * vh;
    }
    if (re(s) > vl) f = f - (T(fl.rail_brake) * m * (s - T(vl))) * vh;
  }
  return f;
}

template <class T>
void apple_loads(const World& W, const OFlags& fl, const Kin<T>& K, const T* ax, const T* av,
                 const int32_t* detached, const int32_t* broken, const double* fext, AppleLoads<T>& A) {
  int na = W.na;
  const std::vector<int> snapped = snapped_bodies(W, broken);
  A.hang.resize(na); A.vhang.resize(na); A.fapp.resize(na); A.a.resize(na);
  A.beta.assign(na, T(0)); A.kappa.assign(na, T(0)); A.tension.resize(na); A.pull.resize(na);
  V3<T> g = dv<T>(W.g);
  const double dt = fl.dt;
  for (int a = 0; a < na; ++a) {
    int b = W.abody[a];
    V3<T> h = K.x[b] + mvec(K.R[b], dv<T>(W.hang + 3 * a));
    A.hang[a] = h;
    A.vhang[a] = K.vx[b] + cross(K.w[b], h - K.x[b]);
    // attached: the state holds the stem elongation u = x - x_hang; detached: the position
    V3<T> ua = {ax[3 * a], ax[3 * a + 1], ax[3 * a + 2]};
    V3<T> va = {av[3 * a], av[3 * a + 1], av[3 * a + 2]};
    V3<T> fs = T(-W.ks[a]) * ua;
    A.tension[a] = sqrt(dot(fs, fs));
    T m = T(W.am[a]);
    const V3<T> fe = rails(fl, m, va, dv<T>(fext + 3 * a));  // the applied force, through the rails
    A.pull[a] = sqrt(dot(fe, fe));
    V3<T> zero = {T(0), T(0), T(0)};
    if (detached[a]) {
      A.fapp[a] = zero;
      A.tension[a] = T(0);
      A.a[a] = va + T(dt) * (g + (T(1) / m) * fe);
      continue;
    }
    T D = m + T(dt * W.cs[a] + dt * dt * W.ks[a]);
    A.a[a] = (T(1) / D) * (m * va + T(dt) * (fe + m * g + fs));
    V3<T> fr = T(-1) * (fs + m * g);
    T n = sqrt(dot(fr, fr));
    double fc = fl.clamp_factor * W.fdet[a];
    if (snapped[b]) {
      // debris: applied forces on a snapped sub-tree are disabled (App. B); the stem still
      // acts on the apple
      A.fapp[a] = zero;
    } else if (fl.tether_implicit) {
      // the clamp scales the coupled reaction, force and stiffness alike, by F_clamp / |f_react|
      T sc = re(n) > fc ? T(fc) / n : T(1);
      A.beta[a] = T(dt * dt * W.ks[a]) / D;
      A.kappa[a] = sc * T(W.ks[a]) * (T(1) - A.beta[a]);
      A.fapp[a] = sc * (fr + T(dt * W.ks[a]) * A.a[a]) - T(dt) * A.kappa[a] * A.vhang[a];
    } else {
      A.fapp[a] = re(n) > fc ? (T(fc) / n) * fr : fr;
    }
  }
}

// M = sum_b m_b Jv_b^T Jv_b + Jw_b^T I_b Jw_b (+ tether terms), dense n_v x n_v.
template <class T>
void mass_matrix(const World& W, const OFlags& fl, const Kin<T>& K, const AppleLoads<T>* A,
                 const int32_t* detached, std::vector<T>& M) {
  int n = W.nv;
  M.assign((size_t)n * n, T(0));
  for (int b = 0; b < W.nb; ++b) {
    const std::vector<int>& ch = W.chain[b];
    M3<T> I = world_inertia(W, K, b);
    T m = T(W.mass[b]);
    for (size_t u = 0; u < ch.size(); ++u) {
      int i = ch[u];
      V3<T> Ji = jac_point(W, K, i, K.c[b]);
      V3<T> IEi = mvec(I, K.e[i]);
      for (size_t v = 0; v < ch.size(); ++v) {
        int j = ch[v];
        V3<T> Jj = jac_point(W, K, j, K.c[b]);
        M[(size_t)i * n + j] += m * dot(Ji, Jj) + dot(K.e[j], IEi);
      }
    }
  }
  if (A) {
    for (int a = 0; a < W.na; ++a) {
      if (detached[a] || re(A->kappa[a]) == 0.0) continue;
      const std::vector<int>& ch = W.chain[W.abody[a]];
      T s = T(fl.dt * fl.dt) * A->kappa[a];
      for (int i : ch)
        for (int j : ch)
          M[(size_t)i * n + j] += s * dot(jac_point(W, K, i, A->hang[a]), jac_point(W, K, j, A->hang[a]));
    }
  }
}

// c(q, qd) = sum_b J_b^T ([m_b (a_c - g); I a + w x I w] - [F_d; tau_d]) - sum_apples J_h^T f_app,
// with the damping wrench of body b at its centre of mass (Sec. IV-A): F_d = -c_v s_b m_b v_c,
// tau_d = -c_omega I_b w_b, where s_b is the snapped factor on a snapped sub-tree (Sec. IV-B:
// "its linear drag is also reduced") and 1 elsewhere. broken: the joints' flags (null: none).
template <class T>
void bias_force(const World& W, const OFlags& fl, const Kin<T>& K, const AppleLoads<T>* A, const int32_t* broken,
                std::vector<T>& c) {
  c.assign(W.nv, T(0));
  V3<T> g = dv<T>(W.g);
  const std::vector<int> snapped = broken ? snapped_bodies(W, broken) : std::vector<int>(W.nb, 0);
  for (int b = 0; b < W.nb; ++b) {
    V3<T> r = K.c[b] - K.x[b];
    V3<T> ac = K.ax[b] + cross(K.al[b], r) + cross(K.w[b], cross(K.w[b], r));
    M3<T> I = world_inertia(W, K, b);
    V3<T> F = T(W.mass[b]) * (ac - g);
    V3<T> N = mvec(I, K.al[b]) + cross(K.w[b], mvec(I, K.w[b]));
    const double cv = fl.lin_damping * (snapped[b] ? fl.snapped_lin_damping : 1.0);
    const V3<T> vc = K.vx[b] + cross(K.w[b], r);
    F = F + T(cv * W.mass[b]) * vc;                 // minus F_d
    N = N + T(fl.ang_damping) * mvec(I, K.w[b]);    // minus tau_d
    for (int i : W.chain[b]) c[i] += dot(jac_point(W, K, i, K.c[b]), F) + dot(K.e[i], N);
  }
  if (A) {
    for (int a = 0; a < W.na; ++a)
      for (int i : W.chain[W.abody[a]]) c[i] -= dot(jac_point(W, K, i, A->hang[a]), A->fapp[a]);
  }
}

// Dense LDL^T solve of the symmetric positive definite H (H x = r), no pivoting.
template <class T> void solve_dense(int n, std::vector<T> H, std::vector<T>& x) {
  std::vector<T> D(n);
  for (int j = 0; j < n; ++j) {
    T s = H[(size_t)j * n + j];
    for (int k = 0; k < j; ++k) s -= H[(size_t)j * n + k] * H[(size_t)j * n + k] * D[k];
    D[j] = s;
    for (int i = j + 1; i < n; ++i) {
      T t = H[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) t -= H[(size_t)i * n + k] * H[(size_t)j * n + k] * D[k];
      H[(size_t)i * n + j] = t / D[j];
    }
  }
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < i; ++k) x[i] -= H[(size_t)i * n + k] * x[k];
  for (int i = 0; i < n; ++i) x[i] /= D[i];
  for (int i = n - 1; i >= 0; --i)
    for (int k = i + 1; k < n; ++k) x[i] -= H[(size_t)k * n + i] * x[k];
}

// Tree-sparse factorisation H = L^T D L with no fill, DOFs eliminated from the leaves to the
// root along the DOF-tree parent array lambda (Featherstone's LTDL), then the two sweeps.
template <class T> void solve_tree(int n, const std::vector<int>& lam, std::vector<T> H, std::vector<T>& x) {
  auto h = [&](int i, int j) -> T& { return H[(size_t)i * n + j]; };
  for (int k = n - 1; k >= 0; --k) {
    int i = lam[k];
    while (i >= 0) {
      T a = h(k, i) / h(k, k);
      int j = i;
      while (j >= 0) {
        h(i, j) -= a * h(k, j);
        j = lam[j];
      }
      h(k, i) = a;
      i = lam[i];
    }
  }
  for (int i = n - 1; i >= 0; --i)
    for (int j = lam[i]; j >= 0; j = lam[j]) x[j] -= h(i, j) * x[i];
  for (int i = 0; i < n; ++i) x[i] /= h(i, i);
  for (int i = 0; i < n; ++i)
    for (int j = lam[i]; j >= 0; j = lam[j]) x[i] -= h(i, j) * x[j];
}

template <class T> struct WState {
  std::vector<T> q, qd, ax, av;
  std::vector<int32_t> broken, bcnt, break_step, detached, pcnt, tcnt, detach_step;
  int32_t status = 0;
};

struct NearLog {
  ORecord* rec;
  std::mutex* mu;
  void add(int w, int kind, int idx, int step, double margin) {
    if (!rec || !rec->near || !rec->near_count) return;
    std::lock_guard<std::mutex> lk(*mu);
    int n = (*rec->near_count)++;
    if (n < rec->near_cap) {
      rec->near[4 * n] = w; rec->near[4 * n + 1] = kind; rec->near[4 * n + 2] = idx; rec->near[4 * n + 3] = step;
      if (rec->near_margin) rec->near_margin[n] = margin;
    }
  }
};

template <class T> bool finite_state(const WState<T>& s) {
  for (const T& v : s.q) if (!std::isfinite(re(v))) return false;
  for (const T& v : s.qd) if (!std::isfinite(re(v))) return false;
  for (const T& v : s.ax) if (!std::isfinite(re(v))) return false;
  for (const T& v : s.av) if (!std::isfinite(re(v))) return false;
  return true;
}

// One step of one world. fext: pull on every apple during this step.
// Per-joint gains in the scalar type (so k and kd can carry complex-step perturbations).
template <class T> struct Gains {
  std::vector<T> k, kd;
};
template <class T> Gains<T> gains_of(const World& W) {
  Gains<T> g;
  for (int b = 0; b < W.nb; ++b) { g.k.push_back(T(W.k[b])); g.kd.push_back(T(W.kd[b])); }
  return g;
}

template <class T>
void step_world(const World& W, const OFlags& fl, WState<T>& s, const Gains<T>& G, const double* fext, int step,
                int widx, NearLog* log) {
  if (s.status & 1) return;  // frozen after a non-finite state
  const double dt = fl.dt;
  Kin<T> K;
  kinematics(W, s.q.data(), s.qd.data(), K);
  for (int a = 0; a < W.na; ++a) {
    if (s.detached[a] != 2) continue;  // detached last step: elongation -> world position
    V3<T> h = K.x[W.abody[a]] + mvec(K.R[W.abody[a]], dv<T>(W.hang + 3 * a));
    s.ax[3 * a] += h.x; s.ax[3 * a + 1] += h.y; s.ax[3 * a + 2] += h.z;
    s.detached[a] = 1;
  }
  AppleLoads<T> A;
  apple_loads(W, fl, K, s.ax.data(), s.av.data(), s.detached.data(), s.broken.data(), fext, A);
  std::vector<T> M, c;
  mass_matrix(W, fl, K, &A, s.detached.data(), M);
  bias_force(W, fl, K, &A, s.broken.data(), c);
  int n = W.nv;
  std::vector<T> r(n);
  for (int i = 0; i < n; ++i) {
    int b = W.dof_body[i];
    // a broken joint loses its spring and its damper (gain rows zeroed, Sec. IV-B); the
    // friction of the torn fibres is introduced at the break and ramped up over break_ramp_s
    // (Sec. IV-B), read as a viscous damper growing from kd to break_ramp_factor * kd
    T k = s.broken[b] ? T(0) : G.k[b];
    T kd = G.kd[b];
    if (s.broken[b]) {
      double since = (step - s.break_step[b]) * dt;
      double ramp = fl.break_ramp_s > 0 ? std::min(since / fl.break_ramp_s, 1.0) : 1.0;
      kd = T(1.0 + (fl.break_ramp_factor - 1.0) * ramp) * G.kd[b];
    }
    M[(size_t)i * n + i] += T(W.arm[b]) + T(dt) * kd + T(fl.alpha_implicit_spring * dt * dt) * k;
    r[i] = T(dt) * (T(-1) * k * (s.q[i] + T(fl.alpha_implicit_spring * dt) * s.qd[i]) - kd * s.qd[i] - c[i]);
  }
  if (n > 0) {
    if (n <= fl.dense_limit) solve_dense(n, M, r);
    else solve_tree(n, W.dof_parent, M, r);
  }
  for (int i = 0; i < n; ++i) {
    s.qd[i] += r[i];
    s.q[i] += T(dt) * s.qd[i];
  }
  // apples (Sec. IV-C): new velocity a + beta v_hang', v_hang' = J_h qd_(n+1) at q_n
  std::vector<int> newly(W.na, 0);
  for (int a = 0; a < W.na; ++a) {
    V3<T> vh = {T(0), T(0), T(0)};
    if (!s.detached[a])
      for (int i : W.chain[W.abody[a]]) vh = vh + s.qd[i] * jac_point(W, K, i, A.hang[a]);
    V3<T> vn = A.a[a] + A.beta[a] * vh;
    V3<T> xa = {s.ax[3 * a], s.ax[3 * a + 1], s.ax[3 * a + 2]};
    // attached: u' = u + dt (v' - v_hang'); detached: x' = x + dt v'
    V3<T> xn = s.detached[a] ? xa + T(dt) * vn : xa + T(dt) * (vn - vh);
    s.ax[3 * a] = xn.x; s.ax[3 * a + 1] = xn.y; s.ax[3 * a + 2] = xn.z;
    s.av[3 * a] = vn.x; s.av[3 * a + 1] = vn.y; s.av[3 * a + 2] = vn.z;
    if (s.detached[a]) continue;
    // detachment tests on this step's pull and tension (Sec. IV-C)
    double P = re(A.pull[a]), Tn = re(A.tension[a]);
    double thr_p = W.fdet[a], thr_t = fl.gamma_tension * W.fdet[a];
    if (log) {
      double mp = std::fabs(P - thr_p) / thr_p, mt = std::fabs(Tn - thr_t) / thr_t;
      if (mp < log->rec->near_eps) log->add(widx, 1, a, step, mp);
      if (mt < log->rec->near_eps) log->add(widx, 2, a, step, mt);
    }
    s.pcnt[a] = P > thr_p ? s.pcnt[a] + 1 : 0;
    s.tcnt[a] = Tn > thr_t ? s.tcnt[a] + 1 : 0;
    if (s.pcnt[a] >= fl.n_pull || s.tcnt[a] >= fl.n_tension) newly[a] = 1;
  }
  // a newly detached apple keeps its elongation until the next step's kinematics turn it
  // into a world position (flag 2)
  for (int a = 0; a < W.na; ++a)
    if (newly[a]) { s.detached[a] = 2; s.detach_step[a] = step; }
  // rupture test on the updated angles: k |theta| > sigma_r pi r^3 / 4 for N_b steps (Eq. 5)
  for (int b = 0; b < W.nb; ++b) {
    if (W.ndof[b] == 0 || s.broken[b]) continue;
    double t2 = 0;
    for (int j = 0; j < W.ndof[b]; ++j) t2 += re(s.q[W.dof0[b] + j]) * re(s.q[W.dof0[b] + j]);
    double mom = re(G.k[b]) * std::sqrt(t2), thr = W.m_max[b];
    if (log) {
      double mg = std::fabs(mom - thr) / thr;
      if (mg < log->rec->near_eps) log->add(widx, 0, b, step, mg);
    }
    s.bcnt[b] = mom > thr ? s.bcnt[b] + 1 : 0;
    if (s.bcnt[b] >= fl.n_break) { s.broken[b] = 1; s.break_step[b] = step; }
  }
  if (!finite_state(s)) s.status |= 1;
}

template <class T> WState<T> load_state(const OForest* f, const OState* st, const World& W, int w) {
  WState<T> s;
  int d0 = dof_offset(f, w), b0 = f->body_off[w], a0 = f->apple_off[w];
  s.q.resize(W.nv); s.qd.resize(W.nv);
  for (int i = 0; i < W.nv; ++i) { s.q[i] = T(st->q[d0 + i]); s.qd[i] = T(st->qd[d0 + i]); }
  s.ax.resize(3 * W.na); s.av.resize(3 * W.na);
  for (int i = 0; i < 3 * W.na; ++i) { s.ax[i] = T(st->ax[3 * a0 + i]); s.av[i] = T(st->av[3 * a0 + i]); }
  s.broken.assign(st->broken + b0, st->broken + b0 + W.nb);
  s.bcnt.assign(st->bcnt + b0, st->bcnt + b0 + W.nb);
  s.break_step.assign(st->break_step + b0, st->break_step + b0 + W.nb);
  s.detached.assign(st->detached + a0, st->detached + a0 + W.na);
  s.pcnt.assign(st->pcnt + a0, st->pcnt + a0 + W.na);
  s.tcnt.assign(st->tcnt + a0, st->tcnt + a0 + W.na);
  s.detach_step.assign(st->detach_step + a0, st->detach_step + a0 + W.na);
  s.status = st->status[w];
  return s;
}

void store_state(const OForest* f, OState* st, const World& W, int w, const WState<double>& s) {
  int d0 = dof_offset(f, w), b0 = f->body_off[w], a0 = f->apple_off[w];
  for (int i = 0; i < W.nv; ++i) { st->q[d0 + i] = s.q[i]; st->qd[d0 + i] = s.qd[i]; }
  for (int i = 0; i < 3 * W.na; ++i) { st->ax[3 * a0 + i] = s.ax[i]; st->av[3 * a0 + i] = s.av[i]; }
  std::copy(s.broken.begin(), s.broken.end(), st->broken + b0);
  std::copy(s.bcnt.begin(), s.bcnt.end(), st->bcnt + b0);
  std::copy(s.break_step.begin(), s.break_step.end(), st->break_step + b0);
  std::copy(s.detached.begin(), s.detached.end(), st->detached + a0);
  std::copy(s.pcnt.begin(), s.pcnt.end(), st->pcnt + a0);
  std::copy(s.tcnt.begin(), s.tcnt.end(), st->tcnt + a0);
  std::copy(s.detach_step.begin(), s.detach_step.end(), st->detach_step + a0);
  st->status[w] = s.status;
}

template <class T> V3<T> tip_point(const World& W, const Kin<T>& K, int t) {
  int b = W.tbody[t];
  return K.x[b] + mvec(K.R[b], dv<T>(W.tlocal + 3 * t));
}

void pulls_at(const World& W, const OPulls* pl, int a0, int step, std::vector<double>& fext) {
  fext.assign(3 * W.na, 0.0);
  if (!pl || !pl->force) return;
  for (int a = 0; a < W.na; ++a) {
    int s0 = pl->start[a0 + a], s1 = pl->end[a0 + a];
    if (step >= s0 && step < s1)
      for (int c = 0; c < 3; ++c) fext[3 * a + c] = pl->force[3 * (a0 + a) + c];
  }
}

void rollout_world(const OForest* f, const OFlags* fl, OState* st, const OPulls* pl, int step0, int n_steps,
                   ORecord* rec, std::mutex* mu, int w) {
  World W = make_world(f, w);
  WState<double> s = load_state<double>(f, st, W, w);
  int a0 = f->apple_off[w], t0 = f->tip_off[w], d0 = dof_offset(f, w);
  int nt_total = f->tip_off[f->n_worlds];
  int nv_total = 0;
  for (int b = 0; b < f->body_off[f->n_worlds]; ++b) nv_total += f->ndof[b];
  NearLog log{rec, mu};
  Gains<double> G = gains_of<double>(W);
  std::vector<double> fext;
  for (int t = 0; t < n_steps; ++t) {
    int step = step0 + t;
    pulls_at(W, pl, a0, step, fext);
    step_world(W, *fl, s, G, fext.data(), step, w, rec ? &log : nullptr);
    if (rec && rec->tips) {
      Kin<double> K;
      kinematics(W, s.q.data(), s.qd.data(), K);
      for (int i = 0; i < W.nt; ++i) {
        V3<double> p = tip_point(W, K, i);
        double* o = rec->tips + ((size_t)t * nt_total + t0 + i) * 3;
        o[0] = p.x; o[1] = p.y; o[2] = p.z;
      }
    }
    if (rec && rec->q)
      for (int i = 0; i < W.nv; ++i) rec->q[(size_t)t * nv_total + d0 + i] = s.q[i];
  }
  store_state(f, st, W, w, s);
}

// Tip-tracking loss of one world over a rollout (reading: sum over steps and tips of
// |p - p*|^2 / (T n_tips)), evaluated in scalar T from a possibly perturbed start.
template <class T>
T world_loss(const World& W, const OFlags& fl, WState<T> s, const Gains<T>& G, const OPulls* pl, int a0, int step0,
             int n_steps, const double* target /* [n_steps][nt][3] world-local tips */) {
  T L = T(0);
  std::vector<double> fext;
  for (int t = 0; t < n_steps; ++t) {
    pulls_at(W, pl, a0, step0 + t, fext);
    step_world(W, fl, s, G, fext.data(), step0 + t, 0, nullptr);
    Kin<T> K;
    kinematics(W, s.q.data(), s.qd.data(), K);
    for (int i = 0; i < W.nt; ++i) {
      V3<T> p = tip_point(W, K, i);
      const double* y = target + ((size_t)t * W.nt + i) * 3;
      V3<T> d = p - dv<T>(y);
      L += dot(d, d);
    }
  }
  return L / T(double(n_steps) * std::max(W.nt, 1));
}

}  // namespace

extern "C" {

// Rollout of every world (in parallel over n_threads host threads).
int oracle_rollout(const OForest* f, const OFlags* fl, OState* st, const OPulls* pl, int step0, int n_steps,
                   ORecord* rec, int n_threads) {
  std::mutex mu;
  int W = f->n_worlds;
  if (n_threads <= 1) {
    for (int w = 0; w < W; ++w) rollout_world(f, fl, st, pl, step0, n_steps, rec, &mu, w);
    return 0;
  }
  std::atomic<int> next(0);
  std::vector<std::thread> th;
  for (int t = 0; t < n_threads; ++t)
    th.emplace_back([&]() {
      for (int w = next++; w < W; w = next++) rollout_world(f, fl, st, pl, step0, n_steps, rec, &mu, w);
    });
  for (auto& t : th) t.join();
  return 0;
}

// Quantities at one configuration of world w (for the pins): dense M (with the tether terms
// when apples are given and the flag is set), bias c (gravity, velocity products, apple
// reactions), body frames, joint origins and centres of mass.
int oracle_eval(const OForest* f, const OFlags* fl, int w, const double* q, const double* qd, const double* ax,
                const double* av, const int32_t* detached, const double* fext, double* M_out, double* c_out,
                double* R_out, double* x_out, double* com_out, double* tension_out, double* fapp_out) {
  World W = make_world(f, w);
  Kin<double> K;
  kinematics(W, q, qd, K);
  std::vector<int32_t> det(W.na, 0);
  if (detached) det.assign(detached, detached + W.na);
  std::vector<double> zeros(3 * W.na, 0.0);
  AppleLoads<double> A;
  apple_loads(W, *fl, K, ax ? ax : zeros.data(), av ? av : zeros.data(), det.data(), nullptr, fext ? fext : zeros.data(), A);
  std::vector<double> M, c;
  mass_matrix(W, *fl, K, ax ? &A : nullptr, det.data(), M);
  bias_force(W, *fl, K, ax ? &A : nullptr, nullptr, c);
  if (M_out) std::copy(M.begin(), M.end(), M_out);
  if (c_out) std::copy(c.begin(), c.end(), c_out);
  for (int b = 0; b < W.nb; ++b) {
    if (R_out) for (int i = 0; i < 9; ++i) R_out[9 * b + i] = K.R[b].a[i];
    if (x_out) { x_out[3 * b] = K.x[b].x; x_out[3 * b + 1] = K.x[b].y; x_out[3 * b + 2] = K.x[b].z; }
    if (com_out) { com_out[3 * b] = K.c[b].x; com_out[3 * b + 1] = K.c[b].y; com_out[3 * b + 2] = K.c[b].z; }
  }
  for (int a = 0; a < W.na; ++a) {
    if (tension_out) tension_out[a] = A.tension[a];
    if (fapp_out) for (int i = 0; i < 3; ++i) fapp_out[3 * a + i] = (&A.fapp[a].x)[i];
  }
  return W.nv;
}

// Solve H x = r for a symmetric positive definite tree-sparse H: mode 0 dense LDL^T,
// mode 1 tree LTDL along the DOF-tree parent array lam.
int oracle_solve(int n, const int32_t* lam, const double* H, double* x, int mode) {
  std::vector<double> Hv(H, H + (size_t)n * n), xv(x, x + n);
  std::vector<int> l(lam, lam + n);
  if (mode == 0) solve_dense(n, Hv, xv);
  else solve_tree(n, l, Hv, xv);
  std::copy(xv.begin(), xv.end(), x);
  return 0;
}

// Loss gradient of one world with respect to selected coordinates, by complex step
// (mode 0; step h, exact to rounding) or central differences (mode 1; per-coordinate
// steps). kinds: 0 = k of body idx, 1 = kd of body idx, 2 = q0[idx], 3 = qd0[idx].
// Masks (break/detach) evolve as in the forward rollout; the caller keeps them frozen by
// choosing a smooth workload.
int oracle_grad(const OForest* f, const OFlags* fl, const OState* st, const OPulls* pl, int w, int step0,
                int n_steps, const double* target, int n_coord, const int32_t* kinds, const int32_t* idx,
                const double* steps, int mode, double* grad, double* loss_out, int n_threads) {
  World W = make_world(f, w);
  int a0 = f->apple_off[w];
  auto one = [&](int ci) -> double {
    int kind = kinds[ci], i = idx[ci];
    double h = steps[ci];
    if (mode == 0) {
      WState<cplx> s = load_state<cplx>(f, st, W, w);
      Gains<cplx> G = gains_of<cplx>(W);
      if (kind == 0) G.k[i] += cplx(0, h);
      if (kind == 1) G.kd[i] += cplx(0, h);
      if (kind == 2) s.q[i] += cplx(0, h);
      if (kind == 3) s.qd[i] += cplx(0, h);
      return std::imag(world_loss<cplx>(W, *fl, s, G, pl, a0, step0, n_steps, target)) / h;
    }
    if (mode == 2) {
      const float hf = (float)h;
      WState<cplxf> s = load_state<cplxf>(f, st, W, w);
      Gains<cplxf> G = gains_of<cplxf>(W);
      if (kind == 0) G.k[i] += cplxf(0, hf);
      if (kind == 1) G.kd[i] += cplxf(0, hf);
      if (kind == 2) s.q[i] += cplxf(0, hf);
      if (kind == 3) s.qd[i] += cplxf(0, hf);
      return (double)std::imag(world_loss<cplxf>(W, *fl, s, G, pl, a0, step0, n_steps, target)) / (double)hf;
    }
    double acc[2];
    for (int sgn = 0; sgn < 2; ++sgn) {
      double d = sgn == 0 ? h : -h;
      WState<double> s = load_state<double>(f, st, W, w);
      Gains<double> G = gains_of<double>(W);
      if (kind == 0) G.k[i] += d;
      if (kind == 1) G.kd[i] += d;
      if (kind == 2) s.q[i] += d;
      if (kind == 3) s.qd[i] += d;
      acc[sgn] = world_loss<double>(W, *fl, s, G, pl, a0, step0, n_steps, target);
    }
    return (acc[0] - acc[1]) / (2 * h);
  };
  if (loss_out) {
    WState<double> s = load_state<double>(f, st, W, w);
    *loss_out = world_loss<double>(W, *fl, s, gains_of<double>(W), pl, a0, step0, n_steps, target);
  }
  std::atomic<int> next(0);
  auto worker = [&]() {
    for (int ci = next++; ci < n_coord; ci = next++) grad[ci] = one(ci);
  };
  int nt = std::max(1, std::min(n_threads, n_coord));
  std::vector<std::thread> th;
  for (int t = 0; t < nt; ++t) th.emplace_back(worker);
  for (auto& t : th) t.join();
  return 0;
}

// Full loss gradient of world w by the reverse-mode scalar (the oracle's own adjoint): dk, dkd
// [nb] and dq0, dqd0 [nv], world-local. Masks follow the plain run. The tape holds every scalar
// operation of the rollout, so this is meant for small worlds and short rollouts: it returns
// -1 (and writes nothing) when the tape would exceed max_nodes.
int oracle_grad_full(const OForest* f, const OFlags* fl, const OState* st, const OPulls* pl, int w, int step0,
                     int n_steps, const double* target, double* dk, double* dkd, double* dq0, double* dqd0,
                     double* loss_out, long long max_nodes) {
  World W = make_world(f, w);
  int a0 = f->apple_off[w];
  Tape tape;
  Tape*& slot = tape_slot();
  Tape* saved = slot;
  slot = &tape;
  WState<RV> s = load_state<RV>(f, st, W, w);
  Gains<RV> G;
  std::vector<int32_t> ik(W.nb), ikd(W.nb), iq(W.nv), iqd(W.nv);
  for (int b = 0; b < W.nb; ++b) {
    G.k.push_back(RV::leaf(W.k[b]));
    ik[b] = G.k.back().id;
    G.kd.push_back(RV::leaf(W.kd[b]));
    ikd[b] = G.kd.back().id;
  }
  for (int i = 0; i < W.nv; ++i) {
    s.q[i] = RV::leaf(s.q[i].v);
    iq[i] = s.q[i].id;
    s.qd[i] = RV::leaf(s.qd[i].v);
    iqd[i] = s.qd[i].id;
  }
  // the tape's size is checked after every step
  RV L = RV(0.0);
  bool over = false;
  {
    std::vector<double> fext;
    for (int t = 0; t < n_steps && !over; ++t) {
      pulls_at(W, pl, a0, step0 + t, fext);
      step_world(W, *fl, s, G, fext.data(), step0 + t, 0, nullptr);
      Kin<RV> K;
      kinematics(W, s.q.data(), s.qd.data(), K);
      for (int i = 0; i < W.nt; ++i) {
        V3<RV> p = tip_point(W, K, i);
        const double* y = target + ((size_t)t * W.nt + i) * 3;
        V3<RV> d = p - dv<RV>(y);
        L += dot(d, d);
      }
      over = (long long)tape.pa.size() > max_nodes;
    }
  }
  if (!over) L = L / RV(double(n_steps) * std::max(W.nt, 1));
  slot = saved;
  if (over) return -1;
  std::vector<double> adj = tape_adjoints(tape, L.id);
  for (int b = 0; b < W.nb; ++b) {
    if (dk) dk[b] = adj[ik[b]];
    if (dkd) dkd[b] = adj[ikd[b]];
  }
  for (int i = 0; i < W.nv; ++i) {
    if (dq0) dq0[i] = adj[iq[i]];
    if (dqd0) dqd0[i] = adj[iqd[i]];
  }
  if (loss_out) *loss_out = L.v;
  return (int)std::min<long long>(tape.pa.size(), 2000000000LL);
}

}  // extern "C"
