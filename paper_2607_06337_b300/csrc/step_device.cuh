// Batched compliant-tree step for sm_103a: one group of TPW threads per world.
//
// Spatial algebra is written in world orientation with each body's own joint origin x_b as
// the reference point (so a hinge's motion subspace is (e_i; 0) and lever arms stay
// segment-sized, which keeps twig inertias well conditioned in FP32). Per step and world:
//   1a. root-to-leaf level sweep: forward kinematics (Sec. IV Eq. 3, two Cardan DOFs per
//       joint), body velocities and velocity-product accelerations (RNE forward pass, base
//       acceleration -g), snapped flags;
//   1b. all bodies at once: the body's spatial inertia, its own Newton-Euler force less the
//       optional body damping (Sec. IV-A), and the apple tether loads (Sec. IV-C Eqs. 6-7, the
//       applied force through the optional rails of App. B), plus the tether coupling point
//       masses;
//   2. leaf-to-root level sweep: RNE force accumulation and CRBA composite inertias; bias
//      c_i = e_i . n_b and the right-hand side r = dt(-K'(q + alpha dt qd) - D' qd - c);
//   3. CRBA rows in ancestor-row storage, body by body, M_ij = e_j . (n_i + (x_b(i) - x_b(j))
//      x f_i) with (n_i; f_i) = I^c_b(i) (e_i; 0), plus the implicit diagonal (armature,
//      dt kd', dt^2 k');
//   4. tree-sparse LDL^T in joint blocks (a joint's one or two DOFs together, see Pivot),
//      level by level from the deepest, each joint a rank-2 update of its ancestor rows; the
//      L^T sweep of the solve rides along; rows are kept unscaled;
//   5. root-to-leaf level sweep: the L sweep of the solve, qd += Delta, q += dt qd, the new
//      body velocities and the rupture tests; then all apples at once: the coupled apple
//      update and the detach tests, with their hysteresis counters (Sec. IV-B Eq. 5,
//      Sec. IV-C).
#pragma once
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>

#include "orchard_dev.h"

// Helpers are __host__ __device__ so the per-world step also compiles for the host (a serial
// group of one thread), which is how its logic is debugged without a GPU.
#define HD __host__ __device__ __forceinline__

namespace orchard {
namespace {

HD float rsq(float x) {
#ifdef __CUDA_ARCH__
  return rsqrtf(x);
#else
  return 1.f / std::sqrt(x);
#endif
}
HD unsigned f2u(float x) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(x);
#else
  unsigned u;
  std::memcpy(&u, &x, 4);
  return u;
#endif
}
HD void atomic_or(unsigned* p, unsigned v) {
#ifdef __CUDA_ARCH__
  atomicOr(p, v);
#else
  *p |= v;
#endif
}
HD void sin_cos(float x, float* s, float* c) {
#ifdef __CUDA_ARCH__
  sincosf(x, s, c);
#else
  *s = std::sin(x);
  *c = std::cos(x);
#endif
}
HD bool finite(float x) {
#ifdef __CUDA_ARCH__
  return isfinite(x);
#else
  return std::isfinite(x);
#endif
}

struct f3 {
  float x, y, z;
};
HD f3 mk(float x, float y, float z) { return {x, y, z}; }
HD f3 operator+(f3 a, f3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
HD f3 operator-(f3 a, f3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
HD f3 operator*(float s, f3 a) { return {s * a.x, s * a.y, s * a.z}; }
HD float dot(f3 a, f3 b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z)); }
HD f3 cross(f3 a, f3 b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
HD f3 ld3(const float* p) { return {p[0], p[1], p[2]}; }
HD void st3(float* p, f3 v) { p[0] = v.x; p[1] = v.y; p[2] = v.z; }
HD f3 xyz(float4 v) { return {v.x, v.y, v.z}; }

// 3x3 rotation, column-major storage c0, c1, c2 (columns are the frame axes).
struct m3 {
  f3 c0, c1, c2;
};
HD f3 mul(const m3& R, f3 v) { return v.x * R.c0 + v.y * R.c1 + v.z * R.c2; }
HD m3 mul(const m3& A, const m3& B) { return {mul(A, B.c0), mul(A, B.c1), mul(A, B.c2)}; }
HD m3 ldm(const float* p) { return {ld3(p), ld3(p + 3), ld3(p + 6)}; }
HD void stm(float* p, const m3& R) { st3(p, R.c0); st3(p + 3, R.c1); st3(p + 6, R.c2); }
HD m3 quat_mat(float4 q) {
  float n = rsq(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
  float w = q.x * n, x = q.y * n, y = q.z * n, z = q.w * n;
  return {mk(1 - 2 * (y * y + z * z), 2 * (x * y + w * z), 2 * (x * z - w * y)),
          mk(2 * (x * y - w * z), 1 - 2 * (x * x + z * z), 2 * (y * z + w * x)),
          mk(2 * (x * z + w * y), 2 * (y * z - w * x), 1 - 2 * (x * x + y * y))};
}

// Symmetric 3x3 (xx, yy, zz, xy, xz, yz) and the 10-number spatial inertia about a point.
struct sym3 {
  float xx, yy, zz, xy, xz, yz;
};
HD f3 mul(const sym3& I, f3 v) {
  return {I.xx * v.x + I.xy * v.y + I.xz * v.z, I.xy * v.x + I.yy * v.y + I.yz * v.z,
          I.xz * v.x + I.yz * v.y + I.zz * v.z};
}
struct sinertia {
  float m;
  f3 h;     // m (com - O)
  sym3 I;   // rotational inertia about O
};
HD void st_in(float* p, const sinertia& s) {
  p[0] = s.m; p[1] = s.h.x; p[2] = s.h.y; p[3] = s.h.z;
  p[4] = s.I.xx; p[5] = s.I.yy; p[6] = s.I.zz; p[7] = s.I.xy; p[8] = s.I.xz; p[9] = s.I.yz;
}
HD sinertia ld_in(const float* p) {
  return {p[0], mk(p[1], p[2], p[3]), {p[4], p[5], p[6], p[7], p[8], p[9]}};
}
// add a point mass mp at offset r from O
HD void add_point(sinertia& s, float mp, f3 r) {
  float rr = dot(r, r);
  s.m += mp;
  s.h = s.h + mp * r;
  s.I.xx += mp * (rr - r.x * r.x); s.I.yy += mp * (rr - r.y * r.y); s.I.zz += mp * (rr - r.z * r.z);
  s.I.xy -= mp * r.x * r.y; s.I.xz -= mp * r.x * r.z; s.I.yz -= mp * r.y * r.z;
}
// add inertia c expressed about O + s (child origin) into acc expressed about O:
// h' = h + m s, I' = I + (2 h.s + m |s|^2) 1 - (h s^T + s h^T) - m s s^T
HD void add_shifted(sinertia& acc, const sinertia& c, f3 s) {
  float hs = dot(c.h, s), ss = dot(s, s);
  float d = 2.f * hs + c.m * ss;
  acc.m += c.m;
  acc.h = acc.h + c.h + c.m * s;
  acc.I.xx += c.I.xx + d - 2.f * c.h.x * s.x - c.m * s.x * s.x;
  acc.I.yy += c.I.yy + d - 2.f * c.h.y * s.y - c.m * s.y * s.y;
  acc.I.zz += c.I.zz + d - 2.f * c.h.z * s.z - c.m * s.z * s.z;
  acc.I.xy += c.I.xy - (c.h.x * s.y + s.x * c.h.y) - c.m * s.x * s.y;
  acc.I.xz += c.I.xz - (c.h.x * s.z + s.x * c.h.z) - c.m * s.x * s.z;
  acc.I.yz += c.I.yz - (c.h.y * s.z + s.y * c.h.z) - c.m * s.y * s.z;
}

template <int TPW>
struct Group {
  int lane;
  int id;      // group index inside the block
  int* flag;   // per-group shared word: 1 once the current world is frozen
  HD void sync() const {
#ifdef __CUDA_ARCH__
    if (TPW == 32) {
      __syncwarp();
    } else {
      asm volatile("bar.sync %0, %1;" ::"r"(id + 1), "r"(TPW) : "memory");
    }
#endif
  }
};

struct WorldView {
  int b0, nb, d0, nv, a0, na, t0, nt, m0, nm, L0, nL, BL0, nBL, f0, nfac, it0, nitem;
  // body-level bounds (nL + 1), factorisation-level bounds, fac_tgt bases and first work
  // items (nBL + 1 each)
  const int *lv, *bb, *bf, *ib;
  // the staged instantiation of the step (ST): the world's table of record pointers (StageTab),
  // written by stage_world. The other instantiation reads the model directly (rec_* below).
  const void* const* tab;
};

// One world's state arrays, indexed world-locally.
struct WState {
  float *q, *qd, *ax, *av;
  int *broken, *bcnt, *break_step, *detached, *pcnt, *tcnt, *detach_step;
  unsigned* status;
};

HD WorldView world_view(const DevModel& m, int w);

HD WState world_state(const DevState& S, const WorldView& v, int w) {
  WState s;
  s.q = S.q + v.d0; s.qd = S.qd + v.d0;
  s.ax = S.ax + 3 * v.a0; s.av = S.av + 3 * v.a0;
  s.broken = S.broken + v.b0; s.bcnt = S.bcnt + v.b0; s.break_step = S.break_step + v.b0;
  s.detached = S.detached + v.a0; s.pcnt = S.pcnt + v.a0; s.tcnt = S.tcnt + v.a0;
  s.detach_step = S.detach_step + v.a0;
  s.status = S.status + w;
  return s;
}

// The state staged in a workspace (WsLayout::S): q, qd (nv, each padded to 4 floats so both
// start on 16-byte boundaries) and the apples' u-or-x, v (3 na) as floats, then broken, bcnt,
// break_step (nb), detached, pcnt, tcnt, detach_step (na) and one status word as ints.
HD WState staged_view(float* base, int nb, int nv, int na) {
  WState s;
  const int nv4 = WsLayout::r4(nv);
  s.q = base; s.qd = base + nv4; s.ax = base + 2 * nv4; s.av = base + 2 * nv4 + 3 * na;
  int* i = (int*)(base + 2 * nv4 + 6 * na);
  s.broken = i; s.bcnt = i + nb; s.break_step = i + 2 * nb;
  s.detached = i + 3 * nb; s.pcnt = s.detached + na; s.tcnt = s.pcnt + na; s.detach_step = s.tcnt + na;
  s.status = (unsigned*)(s.detach_step + na);
  return s;
}

HD WorldView world_view(const DevModel& m, int w) {
  WorldView v;
  v.b0 = m.body_off[w]; v.nb = m.body_off[w + 1] - v.b0;
  v.d0 = m.dof_off[w]; v.nv = m.dof_off[w + 1] - v.d0;
  v.a0 = m.apple_off[w]; v.na = m.apple_off[w + 1] - v.a0;
  v.t0 = m.tip_off[w]; v.nt = m.tip_off[w + 1] - v.t0;
  v.m0 = m.m_off[w]; v.nm = m.m_off[w + 1] - v.m0;
  v.L0 = m.lvl_off[w]; v.nL = m.lvl_off[w + 1] - v.L0 - 1;
  v.BL0 = m.bl_off[w]; v.nBL = m.bl_off[w + 1] - v.BL0 - 1;
  v.f0 = m.fac_off[w];
  v.nfac = m.fac_off[w + 1] - v.f0;
  v.it0 = m.fit_off[w];
  v.nitem = m.fit_off[w + 1] - v.it0;
  v.lv = m.lvl + v.L0;
  v.bb = m.bl_bound + v.BL0;
  v.bf = m.bl_fbase + v.BL0;
  v.ib = m.bl_ibase + v.BL0;
  v.tab = nullptr;
  return v;
}

// A world's model records, world-locally indexed: through the world's table of record pointers
// (ST), else straight from the model (whose pointers are kernel parameters, so they cost no
// registers). The table sits in shared memory: a read costs one shared load and holds nothing.
template <class T> HD const T* tab_ptr(const WorldView& v, int e) { return (const T*)v.tab[e]; }
template <bool ST> HD int4 rec_bi(const DevModel& m, const WorldView& v, int b) {
  return ST ? tab_ptr<int4>(v, kTabBi)[b] : m.bi[v.b0 + b];
}
template <bool ST> HD int4 rec_bj(const DevModel& m, const WorldView& v, int b) {
  return ST ? tab_ptr<int4>(v, kTabBj)[b] : m.bj[v.b0 + b];
}
template <bool ST> HD float4 rec_p0(const DevModel& m, const WorldView& v, int b) {
  return ST ? tab_ptr<float4>(v, kTabP0)[b] : m.bp0[v.b0 + b];
}
template <bool ST> HD float4 rec_p1(const DevModel& m, const WorldView& v, int b) {
  return ST ? tab_ptr<float4>(v, kTabP1)[b] : m.bp1[v.b0 + b];
}
template <bool ST> HD float4 rec_p2(const DevModel& m, const WorldView& v, int b) {
  return ST ? tab_ptr<float4>(v, kTabP2)[b] : m.bp2[v.b0 + b];
}
template <bool ST> HD float4 rec_p3(const DevModel& m, const WorldView& v, int b) {
  return ST ? tab_ptr<float4>(v, kTabP3)[b] : m.bp3[v.b0 + b];
}
template <bool ST> HD float4 rec_p4(const DevModel& m, const WorldView& v, int b) {
  return ST ? tab_ptr<float4>(v, kTabP4)[b] : m.bp4[v.b0 + b];
}
template <bool ST> HD float4 rec_a0(const DevModel& m, const WorldView& v, int a) {
  return ST ? tab_ptr<float4>(v, kTabA0)[a] : m.ap0[v.a0 + a];
}
template <bool ST> HD float4 rec_a1(const DevModel& m, const WorldView& v, int a) {
  return ST ? tab_ptr<float4>(v, kTabA1)[a] : m.ap1[v.a0 + a];
}
template <bool ST> HD int rec_abody(const DevModel& m, const WorldView& v, int a) {
  return ST ? tab_ptr<int>(v, kTabAbody)[a] : m.apple_body[v.a0 + a];
}
template <bool ST> HD int4 rec_info(const DevModel& m, const WorldView& v, int i) {
  return ST ? tab_ptr<int4>(v, kTabInfo)[i] : m.bl_info[v.b0 + i];
}
template <bool ST> HD int4 rec_item(const DevModel& m, const WorldView& v, int i) {
  return ST ? tab_ptr<int4>(v, kTabItems)[i] : m.fitem[v.it0 + i];
}
template <bool ST> HD const unsigned* rec_anc(const DevModel& m, const WorldView& v) {
  return ST ? tab_ptr<unsigned>(v, kTabAnc) : m.anc + v.m0;
}
template <bool ST> HD const int2* rec_fac(const DevModel& m, const WorldView& v) {
  return ST ? tab_ptr<int2>(v, kTabFac) : m.fac_tgt + v.f0;
}

HD f3 apple_force(const StepArgs& a, int ga, int t_abs) {
  f3 f = mk(0.f, 0.f, 0.f);
  if (a.pull_force && t_abs >= a.pull_start[ga] && t_abs < a.pull_end[ga]) f = ld3(a.pull_force + 3 * ga);
  if (a.ext_force) f = f + ld3(a.ext_force + 3 * ga);
  return f;
}

// The rails of App. B on the applied force f of an apple of mass m with velocity v at the
// step's start: (1) impulse cap, the velocity f alone adds in one step is at most v_lim;
// (2) power fade, f's component pushing along v fades linearly from full at |v| = v_fade to
// none at v_lim; (3) speed brake, -c_b m (|v| - v_lim) v / |v| added above v_lim. Rails off
// or no applied force: f unchanged. `tr` (optional) keeps what the adjoint's Jacobian needs.
struct RailTrace {
  f3 f1, vh;        // the force after the cap, v / |v|
  float s, p, phi;  // |v|, f1 . vh, the fade factor
  float dphi;       // d phi / d|v|
  bool fade, brake;
};
HD f3 apply_rails(const StepArgs& a, float m, f3 v, f3 f, RailTrace* tr) {
  RailTrace t;
  t.fade = t.brake = false;
  if (a.rail_v > 0.f) {
    const float fn = sqrtf(dot(f, f));
    if (fn > 0.f) {
      const float cap = m * a.rail_cap;
      if (fn > cap) f = (cap / fn) * f;
      t.f1 = f;
      t.s = sqrtf(dot(v, v));
      if (t.s > a.rail_vf) {
        t.vh = (1.f / t.s) * v;
        t.p = dot(f, t.vh);
        if (t.p > 0.f) {
          t.fade = true;
          t.phi = t.s >= a.rail_v ? 0.f : (a.rail_v - t.s) * a.rail_inv;
          t.dphi = t.s >= a.rail_v ? 0.f : -a.rail_inv;
          f = f - ((1.f - t.phi) * t.p) * t.vh;
        }
        if (t.s > a.rail_v) {
          t.brake = true;
          f = f - (a.rail_cb * m * (t.s - a.rail_v)) * t.vh;
        }
      }
    }
  }
  if (tr) *tr = t;
  return f;
}
// apply_rails out of line, on scalars: keeps the rails' code out of the inlined step, whose
// size costs the backward kernel (which replays the step) even with the rails off.
__host__ __device__ __noinline__ f3 rails_force(float rv, float rvf, float rinv, float rcap, float rcb, float m, f3 v,
                                                f3 f) {
  StepArgs a{};
  a.rail_v = rv;
  a.rail_vf = rvf;
  a.rail_inv = rinv;
  a.rail_cap = rcap;
  a.rail_cb = rcb;
  return apply_rails(a, m, v, f, nullptr);
}

// J^T y with J the Jacobian of apply_rails with respect to v (the force given, the regimes of
// the trace frozen).
HD f3 rails_vjp(const StepArgs& a, float m, const RailTrace& t, f3 y) {
  f3 r = mk(0.f, 0.f, 0.f);
  if (!t.fade && !t.brake) return r;
  const float vy = dot(t.vh, y);
  const f3 yp = y - vy * t.vh;  // (1 - vh vh^T) y
  if (t.fade) {
    const f3 fp = t.f1 - t.p * t.vh;  // (1 - vh vh^T) f1
    r = r + (t.dphi * t.p * vy) * t.vh - ((1.f - t.phi) / t.s) * (vy * fp + t.p * yp);
  }
  if (t.brake) r = r - (a.rail_cb * m) * (vy * t.vh + ((t.s - a.rail_v) / t.s) * yp);
  return r;
}

// The joint damper's factor on kd this step: 1, or for a broken joint the torn-fibre friction,
// a damper growing from kd to (1 + ramp_gain) kd over the ramp time (Sec. IV-B).
HD float damper_factor(const WState& s, const StepArgs& a, int b, int t_abs) {
  if (!s.broken[b]) return 1.f;
  const float since = (float)(t_abs - s.break_step[b]);
  const float ramp = a.ramp_inv > 0.f ? fminf(since * a.ramp_inv, 1.f) : 1.f;
  return 1.f + a.ramp_gain * ramp;
}

// Joint gains of this step: a broken joint has no spring and its damper is scaled by
// damper_factor.
HD void joint_gains(const WState& s, const StepArgs& a, int b, float4 P3, int t_abs, float* k, float* kd) {
  *k = s.broken[b] ? 0.f : P3.z;
  *kd = s.broken[b] ? damper_factor(s, a, b, t_abs) * P3.w : P3.w;
}

// The model records a sweep needs of one body, loaded together (independent addresses, so
// their latencies overlap).
struct KinRec {
  int4 bi;
  float4 P0, P1;
};
template <bool ST>
HD KinRec kin_rec(const DevModel& m, const WorldView& v, int b) {
  return {rec_bi<ST>(m, v, b), rec_p0<ST>(m, v, b), rec_p1<ST>(m, v, b)};
}
struct BwdRec {
  int4 bi;
  float4 P3;
};
template <bool ST>
HD BwdRec bwd_rec(const DevModel& m, const WorldView& v, int b) { return {rec_bi<ST>(m, v, b), rec_p3<ST>(m, v, b)}; }
struct UpdRec {
  int4 bi, bj;
  float4 P3, P4;
};
template <bool ST>
HD UpdRec upd_rec(const DevModel& m, const WorldView& v, int b) {
  return {rec_bi<ST>(m, v, b), rec_bj<ST>(m, v, b), rec_p3<ST>(m, v, b), rec_p4<ST>(m, v, b)};
}
// Phase 1a for one body (root to leaf, level by level): kinematics, velocities, bias
// acceleration, snapped flag.
HD void forward_kin(const WState& s, const WsLayout& L, float* ws, float* sn, int b, f3 g, const KinRec& rec,
                    float* kin) {
  const int4 bi = rec.bi;
  const int p = bi.x;
  const int dof0 = bi.y & 0x0fffffff, nd = (unsigned)bi.y >> 28;
  const float4 P0 = rec.P0, P1 = rec.P1;
  m3 Rp;
  f3 xp, wp, vp, alp, ap;
  if (p >= 0) {
    Rp = ldm(ws + L.R + 9 * p);
    xp = ld3(ws + L.X + 3 * p);
    wp = ld3(ws + L.V + kVel * p); vp = ld3(ws + L.V + kVel * p + 3);
    alp = ld3(ws + L.A + 6 * p); ap = ld3(ws + L.A + 6 * p + 3);
  } else {
    Rp = {mk(1, 0, 0), mk(0, 1, 0), mk(0, 0, 1)};
    xp = wp = vp = alp = mk(0, 0, 0);
    ap = (-1.f) * g;  // gravity as a base acceleration
  }
  m3 R = mul(Rp, quat_mat(P1));
  const f3 xb = xp + mul(Rp, xyz(P0));
  const f3 d = xb - xp;
  const f3 vin = vp + cross(wp, d);
  f3 w = wp, al = alp, aa = ap + cross(alp, d);
  for (int j = 0; j < nd; ++j) {
    const int i = dof0 + j;
    const f3 e = j == 0 ? R.c0 : R.c1;
    st3(ws + L.E + 3 * i, e);
    const float qdj = s.qd[i], qj = s.q[i];
    al = al + qdj * cross(w, e);
    aa = aa + qdj * cross(vin, e);
    w = w + qdj * e;
    float sn, cs;
    sin_cos(qj, &sn, &cs);
    if (j == 0) {  // R <- R Rx(q)
      const f3 c1 = cs * R.c1 + sn * R.c2, c2 = cs * R.c2 - sn * R.c1;
      R.c1 = c1; R.c2 = c2;
    } else {       // R <- R Ry(q)
      const f3 c0 = cs * R.c0 - sn * R.c2, c2 = sn * R.c0 + cs * R.c2;
      R.c0 = c0; R.c2 = c2;
    }
  }
  stm(ws + L.R + 9 * b, R);
  st3(ws + L.X + 3 * b, xb);
  // on a snapped sub-tree (this joint or one above broken): applied forces disabled (App. B)
  const bool snapped = s.broken[b] || (p >= 0 && sn[p] != 0.f);
  sn[b] = snapped ? 1.f : 0.f;
  st3(ws + L.V + kVel * b, w); st3(ws + L.V + kVel * b + 3, vin);
  st3(ws + L.A + 6 * b, al); st3(ws + L.A + 6 * b + 3, aa);
  if (kin) {  // the step's record in the adjoint's tape (WsLayout::kin_offset)
    float4* k4 = reinterpret_cast<float4*>(kin + WsLayout::kKin * b);
    k4[0] = make_float4(R.c0.x, R.c0.y, R.c0.z, R.c1.x);
    k4[1] = make_float4(R.c1.y, R.c1.z, R.c2.x, R.c2.y);
    k4[2] = make_float4(R.c2.z, xb.x, xb.y, xb.z);
    k4[3] = make_float4(w.x, w.y, w.z, vin.x);
    k4[4] = make_float4(vin.y, vin.z, al.x, al.y);
    k4[5] = make_float4(al.z, aa.x, aa.y, aa.z);
  }
}

// Phase 1b for one body (all bodies at once, after 1a): spatial inertia, own Newton-Euler
// force less the body damping, apple loads.
template <bool ST = false>
HD void forward_force(const DevModel& m, const WState& s, const StepArgs& a, const WorldView& v, const WsLayout& L,
                      float* ws, const float* sn, float* atb, int b, int t_abs, f3 g) {
  const int4 bi = rec_bi<ST>(m, v, b);
  const float4 P0 = rec_p0<ST>(m, v, b), P2 = rec_p2<ST>(m, v, b), P3 = rec_p3<ST>(m, v, b);
  const m3 R = ldm(ws + L.R + 9 * b);
  const f3 xb = ld3(ws + L.X + 3 * b);
  const f3 w = ld3(ws + L.V + kVel * b), vin = ld3(ws + L.V + kVel * b + 3);
  const f3 al = ld3(ws + L.A + 6 * b), aa = ld3(ws + L.A + 6 * b + 3);
  const bool snapped = sn[b] != 0.f;

  // spatial inertia of the body about x_b
  const float mb = P0.w;
  const f3 r = mul(R, xyz(P2));
  sinertia I;
  I.m = mb;
  I.h = mb * r;
  {
    const float i0 = P2.w, i1 = P3.x, i2 = P3.y, rr = dot(r, r);
    const f3 c0 = R.c0, c1 = R.c1, c2 = R.c2;
    I.I.xx = i0 * c0.x * c0.x + i1 * c1.x * c1.x + i2 * c2.x * c2.x + mb * (rr - r.x * r.x);
    I.I.yy = i0 * c0.y * c0.y + i1 * c1.y * c1.y + i2 * c2.y * c2.y + mb * (rr - r.y * r.y);
    I.I.zz = i0 * c0.z * c0.z + i1 * c1.z * c1.z + i2 * c2.z * c2.z + mb * (rr - r.z * r.z);
    I.I.xy = i0 * c0.x * c0.y + i1 * c1.x * c1.y + i2 * c2.x * c2.y - mb * r.x * r.y;
    I.I.xz = i0 * c0.x * c0.z + i1 * c1.x * c1.z + i2 * c2.x * c2.z - mb * r.x * r.z;
    I.I.yz = i0 * c0.y * c0.z + i1 * c1.y * c1.z + i2 * c2.y * c2.z - mb * r.y * r.z;
  }
  // own Newton-Euler force at x_b: I (al; aa) + (w; vin) x* I (w; vin)
  const f3 n1 = mul(I.I, al) + cross(I.h, aa), f1 = mb * aa - cross(I.h, al);
  const f3 n2 = mul(I.I, w) + cross(I.h, vin), f2 = mb * vin - cross(I.h, w);
  f3 n = n1 + cross(w, n2) + cross(vin, f2);
  f3 f = f1 + cross(w, f2);
  // velocity-proportional damping at the centre of mass (Sec. IV-A), F = -c_v m v_c (c_v
  // reduced on a snapped sub-tree, Sec. IV-B) and tau = -c_omega I_c w, applied to the body
  if (a.cv != 0.f || a.cw != 0.f) {
    const float kv = (snapped ? a.cv_snap : a.cv) * mb;
    const f3 vc = vin + cross(w, r);
    const f3 wl = mk(dot(R.c0, w), dot(R.c1, w), dot(R.c2, w));
    const f3 Icw = (P2.w * wl.x) * R.c0 + (P3.x * wl.y) * R.c1 + (P3.y * wl.z) * R.c2;
    n = n + a.cw * Icw + kv * cross(r, vc);  // minus (tau + r x F)
    f = f + kv * vc;                          // minus F
  }

  // apples hanging from this body
  const int afirst = bi.w & 0x00ffffff, acount = (unsigned)bi.w >> 24;
  const float dt = a.dt;
  for (int k = 0; k < acount; ++k) {
    const int ai = afirst + k, ga = v.a0 + ai;
    const float4 A0 = rec_a0<ST>(m, v, ai), A1 = rec_a1<ST>(m, v, ai);
    const float ma = A0.w, ks = A1.x, csd = A1.y, fdet = A1.z;
    const f3 rh = mul(R, xyz(A0));
    const f3 xh = xb + rh;
    // attached: the state is the stem elongation u = x - x_hang; detached: the position
    f3 ua = ld3(s.ax + 3 * ai);
    const f3 va = ld3(s.av + 3 * ai);
    int det = s.detached[ai];
    if (det == 2) {  // detached during the last step: elongation -> world position
      ua = ua + xh;
      st3(s.ax + 3 * ai, ua);
      s.detached[ai] = det = 1;
    }
    f3 fe = apple_force(a, ga, t_abs);  // through the rails, when they are on
    if (a.rail_v > 0.f) fe = rails_force(a.rail_v, a.rail_vf, a.rail_inv, a.rail_cap, a.rail_cb, ma, va, fe);
    const f3 fs = det ? mk(0, 0, 0) : (-ks) * ua;
    const float T = sqrtf(dot(fs, fs)), P = sqrtf(dot(fe, fe));
    f3 avec, fapp = mk(0, 0, 0);
    float beta = 0.f, kappa = 0.f;
    if (det) {
      avec = va + dt * (g + (1.f / ma) * fe);
    } else {
      const float D = ma + dt * csd + dt * dt * ks;
      avec = (1.f / D) * (ma * va + dt * (fe + ma * g + fs));
      const f3 fr = (-1.f) * (fs + ma * g);
      const float nfr = sqrtf(dot(fr, fr));
      const float fc = a.clamp * fdet;
      if (snapped) {
        // debris: no reaction on the tree; the stem still acts on the apple
      } else if (a.tether_implicit) {
        // the clamp scales the coupled reaction, force and stiffness alike
        const float sc = nfr > fc ? fc / nfr : 1.f;
        beta = dt * dt * ks / D;
        kappa = sc * ks * (1.f - beta);
        const f3 vh = vin + cross(w, rh);
        fapp = sc * (fr + (dt * ks) * avec) - (dt * kappa) * vh;
      } else {
        fapp = nfr > fc ? (fc / nfr) * fr : fr;
      }
    }
    n = n - cross(rh, fapp);
    f = f - fapp;
    if (kappa > 0.f) add_point(I, dt * dt * kappa, rh);
    float* at = atb + 10 * ai;
    st3(at, avec);
    at[3] = beta; at[4] = T; at[5] = P;
    st3(at + 6, rh);
  }
  st3(ws + L.F + 6 * b, n); st3(ws + L.F + 6 * b + 3, f);
  st_in(ws + L.IC + 10 * b, I);
}

// Phase 2 for one body: pull children, bias and right-hand side of its DOFs.
HD void backward_body(const WState& s, const StepArgs& a, const WsLayout& L, float* ws, int b, int t_abs,
                      const BwdRec& rec) {
  const int4 bi = rec.bi;
  const int dof0 = bi.y & 0x0fffffff, nd = (unsigned)bi.y >> 28;
  const int cfirst = bi.z & 0x00ffffff, ccount = (unsigned)bi.z >> 24;
  f3 n = ld3(ws + L.F + 6 * b), f = ld3(ws + L.F + 6 * b + 3);
  sinertia I = ld_in(ws + L.IC + 10 * b);
  const f3 xb = ld3(ws + L.X + 3 * b);
  for (int k = 0; k < ccount; ++k) {
    const int c = cfirst + k;
    const f3 sft = ld3(ws + L.X + 3 * c) - xb;
    const f3 nc = ld3(ws + L.F + 6 * c), fc = ld3(ws + L.F + 6 * c + 3);
    n = n + nc + cross(sft, fc);
    f = f + fc;
    add_shifted(I, ld_in(ws + L.IC + 10 * c), sft);
  }
  st3(ws + L.F + 6 * b, n); st3(ws + L.F + 6 * b + 3, f);
  st_in(ws + L.IC + 10 * b, I);
  if (nd) {
    float k, kd;
    joint_gains(s, a, b, rec.P3, t_abs, &k, &kd);
    const float dt = a.dt, adt = a.alpha ? dt : 0.f;
    for (int j = 0; j < nd; ++j) {
      const int i = dof0 + j;
      const float c = dot(ld3(ws + L.E + 3 * i), n);
      const float qi = s.q[i], qdi = s.qd[i];
      ws[L.r + i] = dt * (-k * (qi + adt * qdi) - kd * qdi - c);
    }
  }
}

// The factorisation eliminates a joint's DOFs (one or two) together, with the inverse of
// their diagonal block P of H (1x1 or 2x2) taken after every deeper joint is eliminated:
// rows stay unscaled (U), the Schur update of an ancestor pair (i, j) is U_i^T P^-1 U_j, and a
// solve is an L^T sweep leaf to root, the scaling z = P^-1 r, and an L sweep root to leaf
// x = z - P^-1 U x_ancestors. For a two-DOF joint (x, then y'): P = [[H_xx, H_yx], [H_yx, H_yy]]
// and the y' row is the x row shifted by one (its first ancestor is x itself).
struct Pivot {
  float p00, p01, p11;  // P^-1 (symmetric)
};
// Once a level is eliminated the factorisation stores each of its joints' P^-1 in place of the
// block: p00 takes H_xx's place, p11 H_yy's and p01 H_yx's (the y' row's entry of x). The
// later uses (the L sweep, the adjoint's solves) read P^-1 there (pivot_of).
// nd: the joint's DOF count, | 16 to invert the block in FP64 (the thinnest twigs).
HD Pivot invert_block(const float* M, int rowx, int rowy, int nd) {
  Pivot P;
  const float a = M[rowx];
  if ((nd & 3) == 2) {
    const float d = M[rowy], b = M[rowy + 1];
    if (nd & 16) {
      const double inv = 1.0 / ((double)a * d - (double)b * b);
      P.p00 = (float)(d * inv);
      P.p01 = (float)(-b * inv);
      P.p11 = (float)(a * inv);
    } else {
      const float inv = 1.f / (a * d - b * b);
      P.p00 = d * inv;
      P.p01 = -b * inv;
      P.p11 = a * inv;
    }
  } else {
    P.p00 = (nd & 16) ? (float)(1.0 / (double)a) : 1.f / a;
    P.p01 = 0.f;
    P.p11 = 0.f;
  }
  return P;
}
// z = P^-1 r for one joint of a finished level, in place in y, and P^-1 stored in place of the
// joint's block.
HD void scale_and_store(float* M, int4 info, float* y) {
  const Pivot P = invert_block(M, info.y, info.z, info.w);
  const float rx = y[info.x];
  M[info.y] = P.p00;
  if ((info.w & 3) == 2) {
    const float ry = y[info.x + 1];
    y[info.x] = P.p00 * rx + P.p01 * ry;
    y[info.x + 1] = P.p01 * rx + P.p11 * ry;
    M[info.z] = P.p11;
    M[info.z + 1] = P.p01;
  } else {
    y[info.x] = P.p00 * rx;
  }
}
// P^-1 of a joint whose block the factorisation has inverted in place.
HD Pivot pivot_of(const float* M, int rowx, int rowy, int nd) {
  Pivot P;
  P.p00 = M[rowx];
  if ((nd & 3) == 2) {
    P.p11 = M[rowy];
    P.p01 = M[rowy + 1];
  } else {
    P.p01 = 0.f;
    P.p11 = 0.f;
  }
  return P;
}

// z = P^-1 r for one joint, in place in y.
HD void pivot_scale(const float* M, int4 info, float* y) {
  const Pivot P = pivot_of(M, info.y, info.z, info.w);
  const float rx = y[info.x];
  if ((info.w & 3) == 2) {
    const float ry = y[info.x + 1];
    y[info.x] = P.p00 * rx + P.p01 * ry;
    y[info.x + 1] = P.p01 * rx + P.p11 * ry;
  } else {
    y[info.x] = P.p00 * rx;
  }
}

// L sweep of one joint (first DOF dof0, joint record bj as in DevModel::bj): x = z - P^-1 U
// x_ancestors, in place in y (which holds z for this joint and the final x of every ancestor).
template <bool ST = false>
HD void lsweep_joint(const DevModel& m, const WorldView& v, const WsLayout& L, const float* ws, float* y, int dof0,
                     int4 bj) {
  const int nd = bj.w & 3;
  if (nd == 0) return;
  const float* M = ws + L.M;
  const float* rowx = M + bj.x;
  const unsigned* an = rec_anc<ST>(m, v) + bj.x;
  float sx = 0.f, sy = 0.f;
  if (nd == 2) {
    const float* rowy = M + bj.y + 1;  // rowy[c]: the y' row's entry of the x row's c-th ancestor
#pragma unroll 4
    for (int c = 1; c <= bj.z; ++c) {
      const float xa = y[an[c] & 0xffffu];
      sx = fmaf(rowx[c], xa, sx);
      sy = fmaf(rowy[c], xa, sy);
    }
    const Pivot P = pivot_of(M, bj.x, bj.y, bj.w);
    y[dof0] -= P.p00 * sx + P.p01 * sy;
    y[dof0 + 1] -= P.p01 * sx + P.p11 * sy;
  } else {
#pragma unroll 4
    for (int c = 1; c <= bj.z; ++c) sx = fmaf(rowx[c], y[an[c] & 0xffffu], sx);
    y[dof0] -= sx * pivot_of(M, bj.x, -1, bj.w).p00;
  }
}

// Phase 5a for one body (root to leaf, level by level): finish the solve, update, velocities,
// rupture test.
template <bool ST = false>
HD void update_body(const DevModel& m, const WState& s, const StepArgs& a, const WorldView& v, const WsLayout& L,
                    float* ws, int b, int t_abs, int* frozen, const UpdRec& rec) {
  const int4 bi = rec.bi;
  const int p = bi.x;
  const int dof0 = bi.y & 0x0fffffff, nd = (unsigned)bi.y >> 28;
  const float dt = a.dt;
  const f3 xb = ld3(ws + L.X + 3 * b);
  f3 w, vl;
  if (p >= 0) {
    const f3 wp = ld3(ws + L.V + kVel * p), vp = ld3(ws + L.V + kVel * p + 3);
    w = wp;
    vl = vp + cross(wp, xb - ld3(ws + L.X + 3 * p));
  } else {
    w = vl = mk(0, 0, 0);
  }
  bool bad = false;
  float th2 = 0.f;
  lsweep_joint<ST>(m, v, L, ws, ws + L.r, dof0, rec.bj);
  for (int j = 0; j < nd; ++j) {
    const int i = dof0 + j;
    const float x = ws[L.r + i];
    const float qd = s.qd[i] + x;
    const float q = s.q[i] + dt * qd;
    s.qd[i] = qd;
    s.q[i] = q;
    bad |= !finite(q) || !finite(qd);
    th2 = fmaf(q, q, th2);
    w = w + qd * ld3(ws + L.E + 3 * i);
  }
  st3(ws + L.V + kVel * b, w); st3(ws + L.V + kVel * b + 3, vl);

  if (nd && !s.broken[b]) {
    const float mom = rec.P3.z * sqrtf(th2);
    const int cnt = mom > rec.P4.y ? s.bcnt[b] + 1 : 0;
    s.bcnt[b] = cnt;
    if (cnt >= a.n_break) {
      s.broken[b] = 1;
      s.break_step[b] = t_abs;
    }
  }
  if (bad) {
    atomic_or(s.status, 1u);
    *frozen = 1;  // every lane reads it after the group barrier that ends the sweep
  }
}

// Phase 5b for one apple (all apples at once, after the level passes of 5a): the apple update
// with its body's end-of-step velocity, and the detach tests.
template <bool ST = false>
HD void update_apple(const DevModel& m, const WState& s, const StepArgs& a, const WorldView& v, const WsLayout& L,
                     float* ws, const float* atb, int ai, int t_abs, int* frozen) {
  const int b = rec_abody<ST>(m, v, ai);
  const f3 w = ld3(ws + L.V + kVel * b), vl = ld3(ws + L.V + kVel * b + 3);
  const float dt = a.dt;
  const float* at = atb + 10 * ai;
  const bool det = s.detached[ai] != 0;
  const f3 rh = ld3(at + 6);
  const f3 vh = det ? mk(0, 0, 0) : vl + cross(w, rh);
  const f3 vn = ld3(at) + at[3] * vh;
  // attached: u' = u + dt (v' - v_hang'); detached: x' = x + dt v'
  const f3 xn = ld3(s.ax + 3 * ai) + dt * (vn - vh);
  st3(s.av + 3 * ai, vn);
  st3(s.ax + 3 * ai, xn);
  if (!det) {
    const float fdet = rec_a1<ST>(m, v, ai).z;
    const int cp = at[5] > fdet ? s.pcnt[ai] + 1 : 0;
    const int ct = at[4] > a.gamma * fdet ? s.tcnt[ai] + 1 : 0;
    s.pcnt[ai] = cp;
    s.tcnt[ai] = ct;
    if (cp >= a.n_pull || ct >= a.n_tension) {
      s.detached[ai] = 2;  // becomes a world position at the next step's kinematics
      s.detach_step[ai] = t_abs;
    }
  }
  if (!finite(xn.x) || !finite(xn.y) || !finite(xn.z) || !finite(vn.x) || !finite(vn.y) || !finite(vn.z)) {
    atomic_or(s.status, 1u);
    *frozen = 1;  // every lane reads it after the group barrier that ends the pass
  }
}

// Phase 3 for one body: the mass-matrix rows of its DOFs in ancestor-row storage,
// M_ij = e_j . (n_i + (x_b(i) - x_b(j)) x f_i) with (n_i; f_i) = I^c_b(i) (e_i; 0), and the
// implicit diagonal (armature, dt kd', dt^2 k'). The y' row of a two-DOF joint has the x DOF
// (same body, no lever) as its first ancestor and then the x row's, so both rows share one
// walk up the ancestors.
template <bool ST = false>
HD void crba_body(const DevModel& m, const WState& s, const StepArgs& a, const WorldView& v, const WsLayout& L,
                  float* ws, int b, int t_abs, const UpdRec& rec) {
  const int dof0 = rec.bi.y & 0x0fffffff, nd = (unsigned)rec.bi.y >> 28;
  if (nd == 0) return;
  const float dt = a.dt;
  const sinertia I = ld_in(ws + L.IC + 10 * b);
  const f3 xb = ld3(ws + L.X + 3 * b);
  float k, kd;
  joint_gains(s, a, b, rec.P3, t_abs, &k, &kd);
  const float diag = rec.P4.x + dt * kd + (a.alpha ? dt * dt * k : 0.f);
  const f3 ex = ld3(ws + L.E + 3 * dof0);
  const f3 nx = mul(I.I, ex), fx = cross(ex, I.h);
  float* rx = ws + L.M + rec.bj.x;
  const unsigned* an = rec_anc<ST>(m, v) + rec.bj.x;
  rx[0] = dot(ex, nx) + diag;
  if (nd == 2) {
    const f3 ey = ld3(ws + L.E + 3 * (dof0 + 1));
    const f3 ny = mul(I.I, ey), fy = cross(ey, I.h);
    float* ry = ws + L.M + rec.bj.y;
    ry[0] = dot(ey, ny) + diag;
    ry[1] = dot(ex, ny);
#pragma unroll 4
    for (int c = 1; c <= rec.bj.z; ++c) {
      const unsigned ab = an[c];
      const f3 lev = xb - ld3(ws + L.X + 3 * (ab >> 16));
      const f3 ej = ld3(ws + L.E + 3 * (ab & 0xffffu));
      rx[c] = dot(ej, nx + cross(lev, fx));
      ry[c + 1] = dot(ej, ny + cross(lev, fy));
    }
  } else {
#pragma unroll 4
    for (int c = 1; c <= rec.bj.z; ++c) {
      const unsigned ab = an[c];
      const f3 lev = xb - ld3(ws + L.X + 3 * (ab >> 16));
      rx[c] = dot(ld3(ws + L.E + 3 * (ab & 0xffffu)), nx + cross(lev, fx));
    }
  }
}

template <int TPW>
HD void write_ckpt(const WState& s, const StepArgs& a, const WorldView& v, int slot, const Group<TPW>& g) {
  unsigned* base = a.ckpt + (long long)slot * a.ckpt_words;
  unsigned* q = base;
  unsigned* qd = q + a.NV;
  unsigned* ax = qd + a.NV;
  unsigned* av = ax + 3 * a.NA;
  unsigned* br = av + 3 * a.NA;
  unsigned* bc = br + a.NB;
  unsigned* bs = bc + a.NB;
  unsigned* de = bs + a.NB;
  unsigned* pc = de + a.NA;
  unsigned* tc = pc + a.NA;
  for (int i = g.lane; i < v.nv; i += TPW) {
    q[v.d0 + i] = f2u(s.q[i]);
    qd[v.d0 + i] = f2u(s.qd[i]);
  }
  for (int i = g.lane; i < 3 * v.na; i += TPW) {
    ax[3 * v.a0 + i] = f2u(s.ax[i]);
    av[3 * v.a0 + i] = f2u(s.av[i]);
  }
  for (int i = g.lane; i < v.nb; i += TPW) {
    br[v.b0 + i] = s.broken[i];
    bc[v.b0 + i] = s.bcnt[i];
    bs[v.b0 + i] = (unsigned)s.break_step[i];
  }
  for (int i = g.lane; i < v.na; i += TPW) {
    de[v.a0 + i] = s.detached[i];
    pc[v.a0 + i] = s.pcnt[i];
    tc[v.a0 + i] = s.tcnt[i];
  }
}

// Forward kinematics only (positions), for the tip record after the last step.
template <int TPW, bool ST = false>
HD void fk_only(const DevModel& m, const WState& s, const WorldView& v, const WsLayout& L, float* ws,
                        const Group<TPW>& g) {
  for (int l = 0; l < v.nL; ++l) {
    const int lo = v.lv[l], hi = v.lv[l + 1];
    for (int b = lo + g.lane; b < hi; b += TPW) {
      const int4 bi = rec_bi<ST>(m, v, b);
      const int p = bi.x;
      const int dof0 = bi.y & 0x0fffffff, nd = (unsigned)bi.y >> 28;
      m3 Rp;
      f3 xp;
      if (p >= 0) {
        Rp = ldm(ws + L.R + 9 * p);
        xp = ld3(ws + L.X + 3 * p);
      } else {
        Rp = {mk(1, 0, 0), mk(0, 1, 0), mk(0, 0, 1)};
        xp = mk(0, 0, 0);
      }
      m3 R = mul(Rp, quat_mat(rec_p1<ST>(m, v, b)));
      const f3 xb = xp + mul(Rp, xyz(rec_p0<ST>(m, v, b)));
      for (int j = 0; j < nd; ++j) {
        float sn, cs;
        sin_cos(s.q[dof0 + j], &sn, &cs);
        if (j == 0) {
          const f3 c1 = cs * R.c1 + sn * R.c2, c2 = cs * R.c2 - sn * R.c1;
          R.c1 = c1; R.c2 = c2;
        } else {
          const f3 c0 = cs * R.c0 - sn * R.c2, c2 = sn * R.c0 + cs * R.c2;
          R.c0 = c0; R.c2 = c2;
        }
      }
      stm(ws + L.R + 9 * b, R);
      st3(ws + L.X + 3 * b, xb);
    }
    g.sync();
  }
}

template <int TPW>
HD void record_tips(const DevModel& m, const StepArgs& a, const WorldView& v, const WsLayout& L,
                            const float* ws, int slot, const Group<TPW>& g) {
  float* out = a.tips + (long long)slot * a.n_tips_total * 3;
  for (int t = g.lane; t < v.nt; t += TPW) {
    const int b = m.tip_body[v.t0 + t];
    const m3 R = ldm(ws + L.R + 9 * b);
    const f3 p = ld3(ws + L.X + 3 * b) + mul(R, xyz(m.tip_local[v.t0 + t]));
    st3(out + 3 * (v.t0 + t), p);
  }
}

#ifdef __CUDA_ARCH__
// Eight independent segmented scans interleaved, so their shuffle latencies overlap. `span`
// is the longest segment in the warp (warp-uniform): rounds stop once they cover it, since the
// shuffle unit's throughput, not its latency, bounds a block of scanning warps.
__device__ __forceinline__ void seg_scan8(float (&v)[8], int lane, int first, int span) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    if (o >= span) break;
    float t[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) t[j] = __shfl_up_sync(0xffffffffu, v[j], o);
    if (lane - o >= first) {
#pragma unroll
      for (int j = 0; j < 8; ++j) v[j] += t[j];
    }
  }
}

// One segmented scan (span as for seg_scan8).
__device__ __forceinline__ float seg_scan1(float a, int lane, int first, int span) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    if (o >= span) break;
    const float t = __shfl_up_sync(0xffffffffu, a, o);
    if (lane - o >= first) a += t;
  }
  return a;
}

// Four independent segmented scans interleaved (span as for seg_scan8).
__device__ __forceinline__ void seg_scan4(float& a, float& b, float& c, float& d, int lane, int first, int span) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    if (o >= span) break;
    const float ta = __shfl_up_sync(0xffffffffu, a, o);
    const float tb = __shfl_up_sync(0xffffffffu, b, o);
    const float tc = __shfl_up_sync(0xffffffffu, c, o);
    const float td = __shfl_up_sync(0xffffffffu, d, o);
    if (lane - o >= first) {
      a += ta;
      b += tb;
      c += tc;
      d += td;
    }
  }
}
#endif

// Tree-sparse LDL^T of H in joint blocks (see Pivot) with the L^T sweep of the solve fused in.
// All joints of one level (the depth of their first DOF) are eliminated together, deepest first
// (none is another's ancestor, and all their descendants are done). Joint k of level l adds
// -a_c U_k,x[c2] - b_c U_k,y[c2] to entry (anc_c, c2 - c) and -a_c r_x - b_c r_y to r of anc_c,
// for 1 <= c <= c2 <= l, with anc_c the c-th ancestor of k's first DOF and (a_c, b_c) =
// (U_k,x[c], U_k,y[c]) P_k^-1. Listed in depth-first order, the joints of one level that share
// their c-th ancestor are contiguous, so each target's contributions are a segmented sum over
// consecutive lanes: shuffle scans, deterministic, no atomics. Different c means different
// target rows. A 16-warp group works through the level's list of items (c, a run of positions)
// built at upload: a run is cut only between groups that share their c-th ancestor, so no two
// items write the same target, and the warps take the items largest first, in snake order.
// Smaller groups split the c values over their warps, each warp walking all the level's chunks.
// z = P^-1 r is stored once the level is done.
template <int TPW, bool ST = false>
HD void factor_levels(const DevModel& m, const WorldView& v, const WsLayout& L, float* ws, const Group<TPW>& g) {
  float* M = ws + L.M;
  float* r = ws + L.r;
#ifdef __CUDA_ARCH__
  constexpr int NW = TPW / 32;
  const int warp = g.lane >> 5, lane = g.lane & 31;
  for (int l = v.nBL - 1; l >= 0; --l) {
    const int lo = v.bb[l], hi = v.bb[l + 1];
    if (lo == hi) continue;  // no joint has its first DOF at this depth (uniform for the group)
    // Groups of 16 warps take the level's work items (balanced over the warps); smaller groups
    // keep the ancestor distances c split over the warps, each warp walking the level's chunks
    // with its pivots computed once per chunk (measured faster with 4 and 8 warps).
    if (TPW >= 512 && l > 0) {
      const int count = hi - lo;
      const int2* ft = rec_fac<ST>(m, v) + v.bf[l];
      // the level's work items (largest first) dealt to the warps in snake order (round r
      // gives warp w item r NW + w, or r NW + NW - 1 - w when r is odd); each step is one chunk
      // of (up to) 32 positions of an item, and the next step's records are loaded before this
      // one runs
      const int i0 = v.ib[l], i1 = v.ib[l + 1];
      int round = 0;
      int it = i0 + warp;
      int4 item = it < i1 ? rec_item<ST>(m, v, it) : make_int4(1, 0, 0, 0);
      int base = lo + item.y;
      int4 info_n = make_int4(0, 0, 0, 0);
      int2 tk_n = make_int2(0, -1 - lane);
      if (it < i1 && base + lane < lo + item.z) {
        info_n = rec_info<ST>(m, v, base + lane);
        tk_n = ft[(item.x - 1) * count + base + lane - lo];
      }
      while (it < i1) {  // warp-uniform
        const int c = item.x, end = lo + item.z, idx = base + lane;
        const bool valid = idx < end;
        const int4 info = info_n;
        const int2 tk = tk_n;
        // the next step: the item's next chunk, or the warp's next item
        base += 32;
        if (base >= end) {
          ++round;
          it = i0 + round * NW + ((round & 1) ? NW - 1 - warp : warp);
          if (it < i1) {
            item = rec_item<ST>(m, v, it);
            base = lo + item.y;
          }
        }
        info_n = make_int4(0, 0, 0, 0);
        tk_n = make_int2(0, -1 - lane);
        if (it < i1 && base + lane < lo + item.z) {
          info_n = rec_info<ST>(m, v, base + lane);
          tk_n = ft[(item.x - 1) * count + base + lane - lo];
        }
        Pivot P{0.f, 0.f, 0.f};
        float rx = 0.f, ry = 0.f;
        if (valid) {
          P = invert_block(M, info.y, info.z, info.w);
          rx = r[info.x];
          if ((info.w & 3) == 2) ry = r[info.x + 1];
        }
        const bool two = (info.w & 3) == 2;
        const float* rowx = M + info.y;
        const float* rowy = M + (two ? info.z + 1 : info.y);  // rowy[c]: entry of anc_c in the y' row
        const int key = tk.y;
        const int prev = __shfl_up_sync(0xffffffffu, key, 1);
        const int next = __shfl_down_sync(0xffffffffu, key, 1);
        const bool head = lane == 0 || prev != key;
        const bool tail = lane == 31 || next != key;
        const unsigned heads = __ballot_sync(0xffffffffu, head);
        const int first = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
        const int span = __reduce_max_sync(0xffffffffu, (unsigned)(lane - first + 1));
        const float ux = valid ? rowx[c] : 0.f, uy = two ? rowy[c] : 0.f;
        const float ac = ux * P.p00 + uy * P.p01, bc = ux * P.p01 + uy * P.p11;
        float* tgt = M + tk.x;  // entry (anc_c, c2 - c) is tgt[c2]
        int c2 = c;
        for (; c2 + 8 <= l + 1; c2 += 8) {
          float sv[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) sv[j] = valid ? fmaf(ac, rowx[c2 + j], two ? bc * rowy[c2 + j] : 0.f) : 0.f;
          seg_scan8(sv, lane, first, span);
          if (valid && tail) {
#pragma unroll
            for (int j = 0; j < 8; ++j) tgt[c2 + j] -= sv[j];
          }
        }
        // the last up-to-seven entries of the row together with the right-hand side
        const int rem = l + 1 - c2;  // the same for the whole warp
        const float sr = fmaf(ac, rx, bc * ry);
        if (rem <= 3) {
          float s0 = valid && rem > 0 ? fmaf(ac, rowx[c2], two ? bc * rowy[c2] : 0.f) : 0.f;
          float s1 = valid && rem > 1 ? fmaf(ac, rowx[c2 + 1], two ? bc * rowy[c2 + 1] : 0.f) : 0.f;
          float s2 = valid && rem > 2 ? fmaf(ac, rowx[c2 + 2], two ? bc * rowy[c2 + 2] : 0.f) : 0.f;
          float sy = sr;
          seg_scan4(s0, s1, s2, sy, lane, first, span);
          if (valid && tail) {
            if (rem > 0) tgt[c2] -= s0;
            if (rem > 1) tgt[c2 + 1] -= s1;
            if (rem > 2) tgt[c2 + 2] -= s2;
            r[key] -= sy;
          }
        } else {
          float sv[8];
#pragma unroll
          for (int j = 0; j < 7; ++j)
            sv[j] = valid && rem > j ? fmaf(ac, rowx[c2 + j], two ? bc * rowy[c2 + j] : 0.f) : 0.f;
          sv[7] = sr;
          seg_scan8(sv, lane, first, span);
          if (valid && tail) {
#pragma unroll
            for (int j = 0; j < 7; ++j)
              if (rem > j) tgt[c2 + j] -= sv[j];
            r[key] -= sv[7];
          }
        }
      }
    }
    if (TPW < 512 && l > 0) {
      const int count = hi - lo;
      const int2* ft = rec_fac<ST>(m, v) + v.bf[l];
      // the first chunk's joint and first target; later chunks' are loaded one chunk ahead
      int4 info_n = make_int4(0, 0, 0, 0);
      int2 tk_n = make_int2(0, -1 - lane);
      if (lo + lane < hi) {
        info_n = rec_info<ST>(m, v, lo + lane);
        if (1 + warp <= l) tk_n = ft[warp * count + lane];
      }
      for (int base = lo; base < hi; base += 32) {
        const int idx = base + lane;
        const bool valid = idx < hi;
        const int4 info = info_n;
        int2 tk_next = tk_n;
        if (base + 32 + lane < hi) {
          info_n = rec_info<ST>(m, v, base + 32 + lane);
          if (1 + warp <= l) tk_n = ft[warp * count + base + 32 + lane - lo];
        } else {
          info_n = make_int4(0, 0, 0, 0);
          tk_n = make_int2(0, -1 - lane);
        }
        Pivot P{0.f, 0.f, 0.f};
        float rx = 0.f, ry = 0.f;
        if (valid) {
          P = invert_block(M, info.y, info.z, info.w);
          rx = r[info.x];
          if ((info.w & 3) == 2) ry = r[info.x + 1];
        }
        const bool two = (info.w & 3) == 2;
        const float* rowx = M + info.y;
        const float* rowy = M + (two ? info.z + 1 : info.y);  // rowy[c]: entry of anc_c in the y' row
        const int2* fp = ft + (idx - lo);
        // the next target is loaded while the current one is summed
        for (int c = 1 + warp; c <= l; c += NW) {
          const int2 tk = tk_next;
          if (c + NW <= l) tk_next = valid ? fp[(c - 1 + NW) * count] : make_int2(0, -1 - lane);
          const int key = tk.y;
          const int prev = __shfl_up_sync(0xffffffffu, key, 1);
          const int next = __shfl_down_sync(0xffffffffu, key, 1);
          const bool head = lane == 0 || prev != key;
          const bool tail = lane == 31 || next != key;
          const unsigned heads = __ballot_sync(0xffffffffu, head);
          const int first = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
          const int span = __reduce_max_sync(0xffffffffu, (unsigned)(lane - first + 1));
          const float ux = valid ? rowx[c] : 0.f, uy = two ? rowy[c] : 0.f;
          const float ac = ux * P.p00 + uy * P.p01, bc = ux * P.p01 + uy * P.p11;
          float* tgt = M + tk.x;  // entry (anc_c, c2 - c) is tgt[c2]
          int c2 = c;
          for (; c2 + 8 <= l + 1; c2 += 8) {
            float sv[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) sv[j] = valid ? fmaf(ac, rowx[c2 + j], two ? bc * rowy[c2 + j] : 0.f) : 0.f;
            seg_scan8(sv, lane, first, span);
            if (valid && tail) {
#pragma unroll
              for (int j = 0; j < 8; ++j) tgt[c2 + j] -= sv[j];
            }
          }
          // the last up-to-seven entries of the row together with the right-hand side
          const int rem = l + 1 - c2;  // the same for the whole warp
          const float sr = fmaf(ac, rx, bc * ry);
          if (rem <= 3) {
            float s0 = valid && rem > 0 ? fmaf(ac, rowx[c2], two ? bc * rowy[c2] : 0.f) : 0.f;
            float s1 = valid && rem > 1 ? fmaf(ac, rowx[c2 + 1], two ? bc * rowy[c2 + 1] : 0.f) : 0.f;
            float s2 = valid && rem > 2 ? fmaf(ac, rowx[c2 + 2], two ? bc * rowy[c2 + 2] : 0.f) : 0.f;
            float sy = sr;
            seg_scan4(s0, s1, s2, sy, lane, first, span);
            if (valid && tail) {
              if (rem > 0) tgt[c2] -= s0;
              if (rem > 1) tgt[c2 + 1] -= s1;
              if (rem > 2) tgt[c2 + 2] -= s2;
              r[key] -= sy;
            }
          } else {
            float sv[8];
#pragma unroll
            for (int j = 0; j < 7; ++j)
              sv[j] = valid && rem > j ? fmaf(ac, rowx[c2 + j], two ? bc * rowy[c2 + j] : 0.f) : 0.f;
            sv[7] = sr;
            seg_scan8(sv, lane, first, span);
            if (valid && tail) {
#pragma unroll
              for (int j = 0; j < 7; ++j)
                if (rem > j) tgt[c2 + j] -= sv[j];
              r[key] -= sv[7];
            }
          }
        }
      }
    }
    g.sync();
    // z = P^-1 r for this level, and P^-1 stored in place of its block for the later uses
    for (int idx = lo + g.lane; idx < hi; idx += TPW) scale_and_store(M, rec_info<ST>(m, v, idx), r);
  }
  g.sync();
#else
  // one serial lane: the same updates, joint by joint in list order
  for (int l = v.nBL - 1; l >= 0; --l) {
    const int lo = v.bb[l], hi = v.bb[l + 1];
    const int count = hi - lo;
    const int2* ft = rec_fac<ST>(m, v) + v.bf[l];
    for (int idx = lo; idx < hi; ++idx) {
      const int4 info = rec_info<ST>(m, v, idx);
      const bool two = (info.w & 3) == 2;
      const Pivot P = invert_block(M, info.y, info.z, info.w);
      const float rx = r[info.x], ry = two ? r[info.x + 1] : 0.f;
      const float* rowx = M + info.y;
      const float* rowy = M + (two ? info.z + 1 : info.y);
      for (int c = 1; c <= l; ++c) {
        const int2 tk = ft[(c - 1) * count + (idx - lo)];
        const float ux = rowx[c], uy = two ? rowy[c] : 0.f;
        const float ac = ux * P.p00 + uy * P.p01, bc = ux * P.p01 + uy * P.p11;
        for (int c2 = c; c2 <= l; ++c2) M[tk.x + c2] -= fmaf(ac, rowx[c2], two ? bc * rowy[c2] : 0.f);
        r[tk.y] -= fmaf(ac, rx, bc * ry);
      }
    }
    for (int idx = lo; idx < hi; ++idx) scale_and_store(M, rec_info<ST>(m, v, idx), r);
  }
#endif
}

// One step of one world: phases 1-5 of the header comment, ending on a group barrier. When
// tip_slot >= 0 the tips of the state at the start of the step are recorded in that slot.
// Phase clocks of the instrumented build: lane 0 of the group reads the SM clock after each
// phase's closing barrier and adds the elapsed cycles to that phase's counter.
struct PhaseClock {
#ifdef ORCHARD_PHASE_CLOCKS
  long long acc[kPhaseSlots];
  long long t;
  HD void start() {
#ifdef __CUDA_ARCH__
    t = clock64();
#endif
  }
  HD void mark(int i) {
#ifdef __CUDA_ARCH__
    const long long n = clock64();
    acc[i] += n - t;
    t = n;
#endif
  }
#else
  HD void start() {}
  HD void mark(int) {}
#endif
};

template <int TPW, bool ST = false>
HD void step_world(const DevModel& m, const WState& s, const StepArgs& a, const WorldView& v, const WsLayout& L,
                   float* ws, const Group<TPW>& g, int t_abs, f3 gv, int tip_slot, PhaseClock* pc = nullptr,
                   float* kin = nullptr, float* lslot = nullptr) {
  // the snapped flags and the apple records: in the workspace, or (lean placement, lslot) in
  // the group's slot of global memory
  float* sn = lslot ? lslot + WsLayout::lean_sn(v.na) : ws + L.SN;
  // 1. root-to-leaf: kinematics, velocities, own forces, apple loads (and, on a taped step, the
  // kinematics into the step's record at kin)
  for (int l = 0; l < v.nL; ++l) {
    const int lo = v.lv[l], hi = v.lv[l + 1];
    for (int b = lo + g.lane; b < hi; b += TPW) forward_kin(s, L, ws, sn, b, gv, kin_rec<ST>(m, v, b), kin);
    g.sync();
  }
  if (pc) pc->mark(0);
  for (int b = g.lane; b < v.nb; b += TPW)
    forward_force<ST>(m, s, a, v, L, ws, sn, lslot ? lslot : ws + L.AT, b, t_abs, gv);
  g.sync();
  if (pc) pc->mark(1);
  if (tip_slot >= 0) record_tips(m, a, v, L, ws, tip_slot, g);
  if (pc) pc->mark(2);
  // 2. leaf-to-root: forces and composite inertias, right-hand side
  for (int l = v.nL - 1; l >= 0; --l) {
    const int lo = v.lv[l], hi = v.lv[l + 1];
    for (int b = lo + g.lane; b < hi; b += TPW) backward_body(s, a, L, ws, b, t_abs, bwd_rec<ST>(m, v, b));
    g.sync();
  }
  if (pc) pc->mark(3);
  // 3. CRBA rows and the implicit diagonal, body by body
  for (int b = g.lane; b < v.nb; b += TPW) crba_body<ST>(m, s, a, v, L, ws, b, t_abs, upd_rec<ST>(m, v, b));
  g.sync();
  if (pc) pc->mark(4);
  // 4. LDL^T by DOF depth, deepest first, with the L^T sweep of the solve
  factor_levels<TPW, ST>(m, v, L, ws, g);
  if (pc) pc->mark(5);
  // 5. root-to-leaf: L sweep, update, velocities, apples, events
  for (int l = 0; l < v.nL; ++l) {
    const int lo = v.lv[l], hi = v.lv[l + 1];
    for (int b = lo + g.lane; b < hi; b += TPW) update_body<ST>(m, s, a, v, L, ws, b, t_abs, g.flag, upd_rec<ST>(m, v, b));
    g.sync();
  }
  if (pc) pc->mark(6);
  if (v.na > 0) {
    for (int ai = g.lane; ai < v.na; ai += TPW)
      update_apple<ST>(m, s, a, v, L, ws, lslot ? lslot : ws + L.AT, ai, t_abs, g.flag);
    g.sync();
  }
  if (pc) pc->mark(7);
}

// Copy one world's state between two views (group-parallel), status word included.
template <int TPW>
HD void copy_state(const WState& d, const WState& src, const WorldView& v, const Group<TPW>& g) {
  for (int i = g.lane; i < v.nv; i += TPW) {
    d.q[i] = src.q[i];
    d.qd[i] = src.qd[i];
  }
  for (int i = g.lane; i < 3 * v.na; i += TPW) {
    d.ax[i] = src.ax[i];
    d.av[i] = src.av[i];
  }
  for (int i = g.lane; i < v.nb; i += TPW) {
    d.broken[i] = src.broken[i];
    d.bcnt[i] = src.bcnt[i];
    d.break_step[i] = src.break_step[i];
  }
  for (int i = g.lane; i < v.na; i += TPW) {
    d.detached[i] = src.detached[i];
    d.pcnt[i] = src.pcnt[i];
    d.tcnt[i] = src.tcnt[i];
    d.detach_step[i] = src.detach_step[i];
  }
  if (g.lane == 0) *d.status = *src.status;
  g.sync();
}

// Copy n floats (rounded up to whole float4; both ends 16-byte aligned, padding behind both
// regions) from src to dst, group-parallel.
template <int TPW>
HD void copy4(float* dst, const float* src, int n, const Group<TPW>& g) {
#ifdef __CUDA_ARCH__
  if (((reinterpret_cast<uintptr_t>(dst) | reinterpret_cast<uintptr_t>(src)) & 15) != 0) {
    for (int i = g.lane; i < n; i += TPW) dst[i] = src[i];  // not expected: the layouts keep 16-byte alignment
    return;
  }
  const int n4 = (n + 3) >> 2;
  float4* d4 = reinterpret_cast<float4*>(dst);
  const float4* s4 = reinterpret_cast<const float4*>(src);
  // four loads in flight per lane before their stores (the regions do not overlap, but through
  // generic pointers the compiler cannot know it, and would wait out each load in turn)
  int i = g.lane;
  for (; i + 3 * TPW < n4; i += 4 * TPW) {
    const float4 a = s4[i], b = s4[i + TPW], c = s4[i + 2 * TPW], d = s4[i + 3 * TPW];
    d4[i] = a;
    d4[i + TPW] = b;
    d4[i + 2 * TPW] = c;
    d4[i + 3 * TPW] = d;
  }
  for (; i < n4; i += TPW) d4[i] = s4[i];
#else
  for (int i = g.lane; i < n; i += TPW) dst[i] = src[i];
#endif
}
// Copy the parts of the world's model named by `mask` (StagePart) into shared memory at dst
// (StageLayout offsets, after the table) and write the world's table of record pointers at dst:
// each to its copy, or to the model in global memory for a part not staged. Group-parallel, no
// closing barrier: the caller's next group barrier publishes the copies and the table.
template <int TPW>
HD void stage_world(const DevModel& m, WorldView& v, int mask, float* dst, const Group<TPW>& g) {
  const StageLayout S = StageLayout::make(mask, v.nb, v.nm, v.na, v.nfac, v.nitem);
  const void** tab = (const void**)dst;
  // lane e of the group writes entry e (the group has at least kTabEntries lanes)
  auto entry = [&](int e, int off, const void* global) {
    if (g.lane == e) tab[e] = off >= 0 ? (const void*)(dst + off) : global;
  };
  entry(kTabBi, S.bi, m.bi + v.b0);
  entry(kTabBj, S.bj, m.bj + v.b0);
  entry(kTabInfo, S.info, m.bl_info + v.b0);
  entry(kTabP0, S.bp0, m.bp0 + v.b0);
  entry(kTabP1, S.bp1, m.bp1 + v.b0);
  entry(kTabP2, S.bp2, m.bp2 + v.b0);
  entry(kTabP3, S.bp3, m.bp3 + v.b0);
  entry(kTabP4, S.bp4, m.bp4 + v.b0);
  entry(kTabA0, S.ap0, m.ap0 + v.a0);
  entry(kTabA1, S.ap1, m.ap1 + v.a0);
  entry(kTabAnc, S.anc, m.anc + v.m0);
  entry(kTabFac, S.fac, m.fac_tgt + v.f0);
  entry(kTabItems, S.items, m.fitem + v.it0);
  entry(kTabAbody, S.abody, m.apple_body + v.a0);
  v.tab = tab;
  auto rec4 = [&](int off, const void* src, int count) {
    if (off >= 0) copy4<TPW>(dst + off, (const float*)src, 4 * count, g);
  };
  rec4(S.bi, m.bi + v.b0, v.nb);
  rec4(S.bp0, m.bp0 + v.b0, v.nb);
  rec4(S.bp1, m.bp1 + v.b0, v.nb);
  rec4(S.bp3, m.bp3 + v.b0, v.nb);
  rec4(S.bj, m.bj + v.b0, v.nb);
  rec4(S.bp4, m.bp4 + v.b0, v.nb);
  rec4(S.info, m.bl_info + v.b0, v.nb);
  rec4(S.items, m.fitem + v.it0, v.nitem);
  rec4(S.bp2, m.bp2 + v.b0, v.nb);
  rec4(S.ap0, m.ap0 + v.a0, v.na);
  rec4(S.ap1, m.ap1 + v.a0, v.na);
  if (S.anc >= 0) {
    unsigned* d = (unsigned*)(dst + S.anc);
    for (int i = g.lane; i < v.nm; i += TPW) d[i] = m.anc[v.m0 + i];
  }
  if (S.fac >= 0) {
    int2* d = (int2*)(dst + S.fac);
    for (int i = g.lane; i < v.nfac; i += TPW) d[i] = m.fac_tgt[v.f0 + i];
  }
  if (S.abody >= 0) {
    int* d = (int*)(dst + S.abody);
    for (int i = g.lane; i < v.na; i += TPW) d[i] = m.apple_body[v.a0 + i];
  }
}

// Copy one step's record (WsLayout::record_words floats at rec) from the workspace and qd
// (save) or back into them (restore).
template <int TPW>
HD void record_part(float* rec, long long& o, float* ws_part, int n, bool save, const Group<TPW>& g) {
  if (save) copy4<TPW>(rec + o, ws_part, n, g);
  else copy4<TPW>(ws_part, rec + o, n, g);
  o += WsLayout::r4(n);
}
template <int TPW>
HD void record_copy(float* ws, const WsLayout& L, float* qd, const WorldView& v, float* rec, bool save,
                    const Group<TPW>& g) {
  long long o = 0;
  record_part<TPW>(rec, o, ws + L.X, L.E - L.X + 3 * v.nv, save, g);   // X, then E
  record_part<TPW>(rec, o, ws + L.r, L.AT - L.r + 10 * v.na, save, g);  // r, then AT
  record_part<TPW>(rec, o, ws + L.SN, v.nb, save, g);
  record_part<TPW>(rec, o, ws + L.M, v.nm, save, g);
  record_part<TPW>(rec, o, qd, v.nv, save, g);                          // qd at the step's end
  g.sync();
}

// The forward's writes into the adjoint's tape, which covers the last K = tape_steps of the
// rollout's n_steps steps (WsLayout::tape_unit per world and taped step): record false, the
// staged state before step t (t = n_steps: the final state); record true, step t's record.
// Steps before the taped ones write nothing. Not inlined, so that the step loop keeps nothing
// live for it.
template <int TPW>
HD __noinline__ void tape_write(float* tape, const long long* tape_off, int n_steps, int tape_steps, int w, int t,
                                bool record, int nb, int nv, int nm, int na, float* ws, Group<TPW> g) {
  const int k = t - (n_steps - tape_steps);  // index among the taped steps
  if (k < 0) return;
  const WsLayout L = WsLayout::make(nb, nv, nm, na);
  const int snap = WsLayout::snap_words(nb, nv, na);
  float* base = tape + (long long)(tape_steps + 1) * tape_off[w];
  if (!record) {
    copy4<TPW>(base + (long long)k * snap, ws + L.S, snap, g);
    return;
  }
  WorldView v{};
  v.nb = nb; v.nv = nv; v.nm = nm; v.na = na;
  const WState s = staged_view(ws + L.S, nb, nv, na);
  float* rec = base + (long long)(tape_steps + 1) * snap + (long long)k * WsLayout::record_words(nb, nv, nm, na);
  record_copy<TPW>(ws, L, s.qd, v, rec, true, g);  // ends on a group barrier
}

// Where a taped step's kinematics go in the adjoint's tape (the step's record, at
// WsLayout::kin_offset), or null for a step the tape does not cover. Not inlined, as tape_write.
HD __noinline__ float* tape_kin(float* tape, const long long* tape_off, int n_steps, int tape_steps, int w, int t,
                                int nb, int nv, int nm, int na) {
  const int k = t - (n_steps - tape_steps);
  if (k < 0) return nullptr;
  const int snap = WsLayout::snap_words(nb, nv, na);
  float* base = tape + (long long)(tape_steps + 1) * tape_off[w];
  return base + (long long)(tape_steps + 1) * snap + (long long)k * WsLayout::record_words(nb, nv, nm, na) +
         WsLayout::kin_offset(nb, nv, nm, na);
}

// All steps of one world: its state is staged in the workspace for the whole rollout, or with
// the lean placement (lslot: the group's global slot, else null) kept in the state arrays.
template <int TPW, bool ST = false>
HD void run_world(const DevModel& m, const DevState& S, const StepArgs& a, int w, float* ws, float* lslot,
                  const Group<TPW>& g) {
  WorldView v = world_view(m, w);
  const WsLayout L = lslot ? WsLayout::make_lean(v.nb, v.nv, v.nm, v.na) : WsLayout::make(v.nb, v.nv, v.nm, v.na);
  const WState sg = world_state(S, v, w);
  // the state staged in the workspace for the whole rollout, or (lean) read and written where
  // it lives
  const WState s = lslot ? sg : staged_view(ws + L.S, v.nb, v.nv, v.na);
  // the model records this class stages sit after the workspace, for all the world's steps
  if (ST) stage_world<TPW>(m, v, a.stage_mask, ws + a.ws_floats, g);  // launched with a shared workspace
  if (!lslot) copy_state<TPW>(s, sg, v, g);  // ends on a group barrier
  else g.sync();
  const float4 g4 = m.gravity[w];
  const f3 gv = mk(g4.x, g4.y, g4.z);
  if (g.lane == 0) *g.flag = (int)(*s.status & 1u);
  g.sync();
  PhaseClock* pcp = nullptr;
#ifdef ORCHARD_PHASE_CLOCKS
  PhaseClock pc;
  for (int i = 0; i < kPhaseSlots; ++i) pc.acc[i] = 0;
  if (a.phase_clk && g.lane == 0) pcp = &pc;
#endif
  int steps_run = 0;
  for (int t = 0; t < a.n_steps; ++t) {
    if (pcp) pcp->start();
    if (a.ckpt && a.ckpt_every > 0 && t % a.ckpt_every == 0) write_ckpt(s, a, v, t / a.ckpt_every, g);
    if (*g.flag) break;  // frozen after a non-finite state (uniform across the group)
    // the step's first write to the staged state comes after several group barriers
    // (the host never pairs a tape with the lean placement, whose workspace holds no state)
    if (a.tape) tape_write<TPW>(a.tape, m.tape_off, a.n_steps, a.tape_steps, w, t, false, v.nb, v.nv, v.nm, v.na, ws, g);
    if (pcp) pcp->mark(8);
    float* kin = a.tape ? tape_kin(a.tape, m.tape_off, a.n_steps, a.tape_steps, w, t, v.nb, v.nv, v.nm, v.na)
                        : nullptr;
    step_world<TPW, ST>(m, s, a, v, L, ws, g, a.step0 + t, gv, (a.tips && t > 0) ? t - 1 : -1, pcp, kin, lslot);
    if (a.tape) tape_write<TPW>(a.tape, m.tape_off, a.n_steps, a.tape_steps, w, t, true, v.nb, v.nv, v.nm, v.na, ws, g);
    if (pcp) pcp->mark(8);
    ++steps_run;
  }
#ifdef ORCHARD_PHASE_CLOCKS
#ifdef __CUDA_ARCH__
  if (pcp) {
    for (int i = 0; i < kPhases; ++i) atomicAdd(a.phase_clk + i, (unsigned long long)pc.acc[i]);
    atomicAdd(a.phase_clk + kPhases, (unsigned long long)steps_run);
  }
#endif
#endif
  (void)steps_run;
  // the final state (its status word tells the backward whether the world froze)
  if (a.tape)
    tape_write<TPW>(a.tape, m.tape_off, a.n_steps, a.tape_steps, w, a.n_steps, false, v.nb, v.nv, v.nm, v.na, ws, g);
  if (a.tips && a.n_steps > 0) {
    fk_only<TPW, ST>(m, s, v, L, ws, g);
    record_tips(m, a, v, L, ws, a.n_steps - 1, g);
    g.sync();
  }
  if (!lslot) copy_state<TPW>(sg, s, v, g);
  else g.sync();
}

}  // namespace
}  // namespace orchard
