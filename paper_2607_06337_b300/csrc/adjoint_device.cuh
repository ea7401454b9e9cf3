// Adjoint of the batched compliant-tree step (device code, also compilable for the host as a
// serial group). Masks (breaks, detachments) are frozen as the forward recorded them.
//
// One step maps (q, qd, u, v) to (q', qd', u', v') through Delta = H^-1 r, qd' = qd + Delta,
// q' = q + dt qd', and the coupled apple update. With Delta-bar the cotangent of Delta and
// lambda = H^-1 Delta-bar, the cotangents of the step inputs are the direct terms of the update
// equations plus the gradient, with Delta held fixed, of
//   psi = lambda^T (r - H Delta)
//       = -dt sum_i lambda_i [k'_i (q_i + alpha dt qd'_i) + kd'_i qd'_i]
//         - dt lambda^T ID(q, qd, Delta / dt)
//         + dt sum_apples [ w_a . P0_a - dt kappa_a w_a . v_hang'_a ],
// where ID is the inverse dynamics (inertia, velocity products, gravity, less the optional body
// damping), w_a = J_h lambda is the virtual velocity of the hang point and P0_a the clamped
// reaction of the coupled tether (with the applied force through the optional rails, whose
// dependence on the apple's velocity is taken in rails_adjoint).
// lambda^T ID = sum_b Lambda_b . F_b (virtual work of each body's Newton-Euler force under the
// virtual velocity Lambda_b of lambda), so the q and qd gradients come from one reverse sweep
// over a per-body tape of the forward kinematics, velocities, accelerations and the virtual
// velocities of lambda and of qd'. Tip cotangents enter as point loads at the configuration
// they were recorded in.
#pragma once
#include "step_device.cuh"

namespace orchard {
namespace {

HD float u2f(unsigned u) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float x;
  std::memcpy(&x, &u, 4);
  return x;
#endif
}

// Fixed-size records (N floats, N a multiple of 4, starting on a 16-byte boundary) moved as
// float4 on the device.
template <int N>
HD void ld_rec(const float* src, float (&d)[N]) {
#ifdef __CUDA_ARCH__
  const float4* s4 = reinterpret_cast<const float4*>(src);
#pragma unroll
  for (int i = 0; i < N / 4; ++i) {
    const float4 v = s4[i];
    d[4 * i] = v.x; d[4 * i + 1] = v.y; d[4 * i + 2] = v.z; d[4 * i + 3] = v.w;
  }
#else
  for (int i = 0; i < N; ++i) d[i] = src[i];
#endif
}
template <int N>
HD void st_rec(float* dst, const float (&v)[N]) {
#ifdef __CUDA_ARCH__
  float4* d4 = reinterpret_cast<float4*>(dst);
#pragma unroll
  for (int i = 0; i < N / 4; ++i) d4[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
#else
  for (int i = 0; i < N; ++i) dst[i] = v[i];
#endif
}
HD void put3(float* r, int o, f3 v) { r[o] = v.x; r[o + 1] = v.y; r[o + 2] = v.z; }
HD f3 get3(const float* r, int o) { return mk(r[o], r[o + 1], r[o + 2]); }
HD m3 getm(const float* r, int o) { return {get3(r, o), get3(r, o + 3), get3(r, o + 6)}; }

// Backward temporaries of one world (floats), at their own base `wa` (shared or global
// memory), and the snapshots of one checkpoint segment (global memory, `seg`). The per-DOF and
// per-apple arrays come first (`small` floats), then the tape T, then the C slots: the arrays
// before T, or before C (`head`), may live in shared memory while the rest stays in global
// memory. T is reached through `tb` (set by backward_world: wa + T, or its own base), C through
// RevArgs::cs.
struct AdjLayout {
  int T;          // tape, 36 per body: R, x, w, v, alpha, a, Lw, Lv, Ow, Ov (see tape_body)
  int C;          // 44 per body: cotangents a body sends to its parent's tape outputs (36),
                  // the hang-velocity channel of Ow, Ov (6; it feeds q, not qd), 2 of padding
  int AF;         // 6 per body: force sweep accumulator
  int qb, qdb;    // per DOF: cotangents of the step-start q, qd being built
  int qb1, qdb1;  // per DOF: cotangents of the step-end q', qd'
  int lam;        // per DOF: lambda (first Delta-bar)
  int qd1;        // per DOF: qd' of the step being reversed
  int zero;       // per DOF: zeros
  int ub, vb;     // per apple x3: cotangents of the step-start u (or x), v
  int ub1, vb1;   // per apple x3: of the step-end u', v'
  int vh;         // per apple x3: cotangent of the new hang-point velocity
  int small;      // floats before T
  int head;       // floats before C
  int total;      // floats at wa
  int snap;       // words per snapshot: the private state, staged in the forward workspace
  float* tb;      // the tape T of the world being reversed
  HD static AdjLayout make(int nb, int nv, int na) {
    // every array starts on a 16-byte boundary
    AdjLayout A;
    int o = 0;
    A.AF = o; o += WsLayout::r4(6 * nb);
    A.qb = o; o += WsLayout::r4(nv);
    A.qdb = o; o += WsLayout::r4(nv);
    A.qb1 = o; o += WsLayout::r4(nv);
    A.qdb1 = o; o += WsLayout::r4(nv);
    A.lam = o; o += WsLayout::r4(nv);
    A.qd1 = o; o += WsLayout::r4(nv);
    A.zero = o; o += WsLayout::r4(nv);
    A.ub = o; o += WsLayout::r4(3 * na);
    A.vb = o; o += WsLayout::r4(3 * na);
    A.ub1 = o; o += WsLayout::r4(3 * na);
    A.vb1 = o; o += WsLayout::r4(3 * na);
    A.vh = o; o += WsLayout::r4(3 * na);
    A.small = o;
    A.T = o; o += 36 * nb;
    A.head = o;
    A.C = o; o += 44 * nb;
    A.snap = WsLayout::snap_words(nb, nv, na);
    A.total = o;
    A.tb = nullptr;
    return A;
  }
};

// Copy the private state (staged at ws + L.S) to or from snapshot `k` of the segment buffer.
template <int TPW>
HD void snapshot(float* ws, const WsLayout& L, float* seg, const AdjLayout& A, int k, bool save, const Group<TPW>& g) {
  float* st = ws + L.S;
  float* sn = seg + (long long)k * A.snap;
  if (save) copy4<TPW>(sn, st, A.snap, g);
  else copy4<TPW>(st, sn, A.snap, g);
  g.sync();
}

// One step's record (WsLayout::record_words): saved by the forward rollout into its tape, or
// by the backward during a checkpoint segment's replay, so that the step's reverse need not
// run the step again.
template <int TPW>
HD void step_record(float* ws, const WsLayout& L, const WState& s, float* wa, const AdjLayout& A,
                    const WorldView& v, float* rec, bool save, const Group<TPW>& g) {
  record_copy<TPW>(ws, L, save ? s.qd : wa + A.qd1, v, rec, save, g);
}

// Load checkpoint `slot` of the forward record into the private state (its world's ranges).
template <int TPW>
HD void load_ckpt(const StepArgs& a, const WorldView& v, const WState& s, int slot, const Group<TPW>& g) {
  const unsigned* base = a.ckpt + (long long)slot * a.ckpt_words;
  const unsigned* q = base;
  const unsigned* qd = q + a.NV;
  const unsigned* ax = qd + a.NV;
  const unsigned* av = ax + 3 * a.NA;
  const unsigned* br = av + 3 * a.NA;
  const unsigned* bc = br + a.NB;
  const unsigned* bs = bc + a.NB;
  const unsigned* de = bs + a.NB;
  const unsigned* pc = de + a.NA;
  const unsigned* tc = pc + a.NA;
  for (int i = g.lane; i < v.nv; i += TPW) {
    s.q[i] = u2f(q[v.d0 + i]);
    s.qd[i] = u2f(qd[v.d0 + i]);
  }
  for (int i = g.lane; i < 3 * v.na; i += TPW) {
    s.ax[i] = u2f(ax[3 * v.a0 + i]);
    s.av[i] = u2f(av[3 * v.a0 + i]);
  }
  for (int i = g.lane; i < v.nb; i += TPW) {
    s.broken[i] = (int)br[v.b0 + i];
    s.bcnt[i] = (int)bc[v.b0 + i];
    s.break_step[i] = (int)bs[v.b0 + i];
  }
  for (int i = g.lane; i < v.na; i += TPW) {
    s.detached[i] = (int)de[v.a0 + i];
    s.pcnt[i] = (int)pc[v.a0 + i];
    s.tcnt[i] = (int)tc[v.a0 + i];
    s.detach_step[i] = -1;
  }
  if (g.lane == 0) *s.status = 0u;
  g.sync();
}

// Tape of one body: forward kinematics at q, body velocity (w, v at x_b), full spatial
// acceleration (alpha, a) with qdd = Delta / dt, and the virtual velocities of lambda (Lw, Lv)
// and of qd' (Ow, Ov).
HD void tape_body(const DevModel& m, const WState& s, const WorldView& v, const AdjLayout& A, float* wa,
                  const float* delta, float inv_dt, const float* lam, const float* qd1, int b, f3 g) {
  const int gb = v.b0 + b;
  const int4 bi = m.bi[gb];
  const int p = bi.x;
  const int dof0 = bi.y & 0x0fffffff, nd = (unsigned)bi.y >> 28;
  m3 Rp;
  f3 xp, wp, vp, alp, ap, lwp, lvp, owp, ovp;
  if (p >= 0) {
    float tp[36];
    ld_rec(A.tb + 36 * p, tp);
    Rp = getm(tp, 0);
    xp = get3(tp, 9); wp = get3(tp, 12); vp = get3(tp, 15); alp = get3(tp, 18); ap = get3(tp, 21);
    lwp = get3(tp, 24); lvp = get3(tp, 27); owp = get3(tp, 30); ovp = get3(tp, 33);
  } else {
    Rp = {mk(1, 0, 0), mk(0, 1, 0), mk(0, 0, 1)};
    xp = wp = vp = alp = lwp = lvp = owp = ovp = mk(0, 0, 0);
    ap = (-1.f) * g;
  }
  m3 R = mul(Rp, quat_mat(m.bp1[gb]));
  const f3 xb = xp + mul(Rp, xyz(m.bp0[gb]));
  const f3 d = xb - xp;
  const f3 vin = vp + cross(wp, d), lvin = lvp + cross(lwp, d), ovin = ovp + cross(owp, d);
  f3 w = wp, al = alp, aa = ap + cross(alp, d), lw = lwp, ow = owp;
  for (int j = 0; j < nd; ++j) {
    const int i = dof0 + j;
    const f3 e = j == 0 ? R.c0 : R.c1;
    al = al + s.qd[i] * cross(w, e) + (delta[i] * inv_dt) * e;
    aa = aa + s.qd[i] * cross(vin, e);
    w = w + s.qd[i] * e;
    lw = lw + lam[i] * e;
    ow = ow + qd1[i] * e;
    float sn, cs;
    sin_cos(s.q[i], &sn, &cs);
    if (j == 0) {
      const f3 c1 = cs * R.c1 + sn * R.c2, c2 = cs * R.c2 - sn * R.c1;
      R.c1 = c1; R.c2 = c2;
    } else {
      const f3 c0 = cs * R.c0 - sn * R.c2, c2 = sn * R.c0 + cs * R.c2;
      R.c0 = c0; R.c2 = c2;
    }
  }
  float t[36];
  put3(t, 0, R.c0); put3(t, 3, R.c1); put3(t, 6, R.c2);
  put3(t, 9, xb); put3(t, 12, w); put3(t, 15, vin); put3(t, 18, al); put3(t, 21, aa);
  put3(t, 24, lw); put3(t, 27, lvin); put3(t, 30, ow); put3(t, 33, ovin);
  st_rec(A.tb + 36 * b, t);
}

// tape_body for a step with a record: the kinematics come from the record's kinematic part
// (kin: R, x_b, w, v at x_b and the velocity-product accelerations, as the forward's kinematics
// sweep found them), so only the parts linear in Delta, lambda and qd' are swept here. The joint
// accelerations qdd = Delta / dt add alpha_D = alpha_D,p + sum_j qdd_j e_j and a_D = a_D,p +
// alpha_D,p x d on top of the record's accelerations; the parent's parts come back as its tape's
// accelerations less its record's. The DOF axes e are the step's (restored at L.E).
HD void tape_body_recorded(const DevModel& m, const WorldView& v, const WsLayout& L, const AdjLayout& A,
                           const float* ws, float* wa, const float* delta, float inv_dt, const float* lam,
                           const float* qd1, int b, const float* kin) {
  const int4 bi = m.bi[v.b0 + b];
  const int p = bi.x;
  const int dof0 = bi.y & 0x0fffffff, nd = (unsigned)bi.y >> 28;
  float k[WsLayout::kKin];
  ld_rec(kin + WsLayout::kKin * b, k);
  const f3 xb = get3(k, 9);
  f3 xp, ald, aad, lw, lvp, ow, ovp;
  if (p >= 0) {
    float tp[36];
    ld_rec(A.tb + 36 * p, tp);
    const float4* kp = reinterpret_cast<const float4*>(kin + WsLayout::kKin * p);
    const float4 k4 = kp[4], k5 = kp[5];  // the parent's record: al (k4.z, k4.w, k5.x), a (k5.yzw)
    xp = get3(tp, 9);
    ald = get3(tp, 18) - mk(k4.z, k4.w, k5.x);
    aad = get3(tp, 21) - mk(k5.y, k5.z, k5.w);
    lw = get3(tp, 24); lvp = get3(tp, 27); ow = get3(tp, 30); ovp = get3(tp, 33);
  } else {
    xp = ald = aad = lw = lvp = ow = ovp = mk(0, 0, 0);
  }
  const f3 d = xb - xp;
  const f3 lvin = lvp + cross(lw, d), ovin = ovp + cross(ow, d);
  aad = aad + cross(ald, d);
  for (int j = 0; j < nd; ++j) {
    const int i = dof0 + j;
    const f3 e = ld3(ws + L.E + 3 * i);
    ald = ald + (delta[i] * inv_dt) * e;
    lw = lw + lam[i] * e;
    ow = ow + qd1[i] * e;
  }
  float t[36];
#pragma unroll
  for (int j = 0; j < 18; ++j) t[j] = k[j];  // R, x_b, w, v at x_b
  put3(t, 18, get3(k, 18) + ald); put3(t, 21, get3(k, 21) + aad);
  put3(t, 24, lw); put3(t, 27, lvin); put3(t, 30, ow); put3(t, 33, ovin);
  st_rec(A.tb + 36 * b, t);
}

// Reverse of a 3x3 symmetric-product term: G accumulates d(phi)/d(Io) as a general matrix.
struct g33 {
  f3 c0, c1, c2;  // columns
};
HD void g_add_outer(g33& G, f3 u, f3 v) {  // G += u v^T
  G.c0 = G.c0 + v.x * u; G.c1 = G.c1 + v.y * u; G.c2 = G.c2 + v.z * u;
}
HD f3 g_mulT_plus(const g33& G, f3 x) {  // (G + G^T) x
  const f3 gx = x.x * G.c0 + x.y * G.c1 + x.z * G.c2;
  const f3 gtx = mk(dot(G.c0, x), dot(G.c1, x), dot(G.c2, x));
  return gx + gtx;
}

struct RevArgs {
  int dyn;               // 1: include the step's dynamics terms; 0: only tip / point seeds
  const float* delta;    // per DOF: the step's Delta
  const float* lam;      // per DOF
  const float* qd1;      // per DOF: qd'
  const float* tipbar;   // [n_tips_total][3] cotangents of this configuration's tips, or null
  float sphi;            // scale of the virtual-work term (-dt)
  float* cs;             // the C slots, 44 floats per body
};

// The cotangent of one body's tape outputs, in a C slot's layout: R (9), x_b, w, v, alpha,
// a, Lw, Lv, Ow, Ov (3 each), then the hang-point channel Ow_h, Ov_h: cotangents of J_h qd'
// seen by the apple update, whose qd' part is already in Delta-bar (hang_load_sweep), so this
// channel only reaches q (through the axes and hang offsets).
struct Cot {
  m3 R;
  f3 x, w, v, al, a, lw, lv, ow, ov, owh, ovh;
};
HD Cot cot_get(const float* c) {
  return {{mk(c[0], c[1], c[2]), mk(c[3], c[4], c[5]), mk(c[6], c[7], c[8])},
          get3(c, 9), get3(c, 12), get3(c, 15), get3(c, 18), get3(c, 21), get3(c, 24), get3(c, 27),
          get3(c, 30), get3(c, 33), get3(c, 36), get3(c, 39)};
}
HD void cot_put(float* c, const Cot& k) {
  put3(c, 0, k.R.c0); put3(c, 3, k.R.c1); put3(c, 6, k.R.c2);
  put3(c, 9, k.x); put3(c, 12, k.w); put3(c, 15, k.v); put3(c, 18, k.al); put3(c, 21, k.a);
  put3(c, 24, k.lw); put3(c, 27, k.lv); put3(c, 30, k.ow); put3(c, 33, k.ov);
  put3(c, 36, k.owh); put3(c, 39, k.ovh);
  c[42] = 0.f;
  c[43] = 0.f;
}

// The reverse of one body's tape runs in two parts. reverse_seed (all bodies at once): the
// cotangents its own terms put on its tape outputs (the virtual work of its Newton-Euler
// force, its apples, its tips), which depend on nothing below it; they are additive, so they
// go into its C slot before the leaf-to-root sweep. reverse_chain (leaf to root): adds the
// children's C slots, reverses the body's DOF loop and its shift from the parent, and leaves
// what goes to the parent in its C slot.
HD void reverse_seed(const DevModel& m, const WState& s, const StepArgs& a, const WorldView& v, const WsLayout& L,
                     const AdjLayout& A, float* ws, float* wa, const RevArgs& ra, int b, f3 g, int t_abs) {
  const int gb = v.b0 + b;
  const int4 bi = m.bi[gb];
  const float dt = a.dt;
  m3 Rb_ = {mk(0, 0, 0), mk(0, 0, 0), mk(0, 0, 0)};
  f3 xbb = mk(0, 0, 0), wb_ = xbb, vb_ = xbb, alb = xbb, ab_ = xbb, lwb = xbb, lvb = xbb, owb = xbb, ovb = xbb;
  f3 owh = xbb, ovh = xbb;

  // own forward values
  float t[36];
  ld_rec(A.tb + 36 * b, t);
  const m3 R = getm(t, 0);
  const f3 w = get3(t, 12), vin = get3(t, 15), al = get3(t, 18), aa = get3(t, 21);
  const f3 lw = get3(t, 24), lv = get3(t, 27), ow = get3(t, 30), ov = get3(t, 33);

  // seeds: virtual work of the body's own Newton-Euler force
  if (ra.dyn) {
    const float4 P0 = m.bp0[gb], P2 = m.bp2[gb], P3 = m.bp3[gb];
    const float mb = P0.w;
    const f3 com = xyz(P2);
    const float Di[3] = {P2.w, P3.x, P3.y};
    const f3 r = mul(R, com);
    const f3 h = mb * r;
    sym3 Io;
    {
      const float rr = dot(r, r);
      const f3 c0 = R.c0, c1 = R.c1, c2 = R.c2;
      Io.xx = Di[0] * c0.x * c0.x + Di[1] * c1.x * c1.x + Di[2] * c2.x * c2.x + mb * (rr - r.x * r.x);
      Io.yy = Di[0] * c0.y * c0.y + Di[1] * c1.y * c1.y + Di[2] * c2.y * c2.y + mb * (rr - r.y * r.y);
      Io.zz = Di[0] * c0.z * c0.z + Di[1] * c1.z * c1.z + Di[2] * c2.z * c2.z + mb * (rr - r.z * r.z);
      Io.xy = Di[0] * c0.x * c0.y + Di[1] * c1.x * c1.y + Di[2] * c2.x * c2.y - mb * r.x * r.y;
      Io.xz = Di[0] * c0.x * c0.z + Di[1] * c1.x * c1.z + Di[2] * c2.x * c2.z - mb * r.x * r.z;
      Io.yz = Di[0] * c0.y * c0.z + Di[1] * c1.y * c1.z + Di[2] * c2.y * c2.z - mb * r.y * r.z;
    }
    const f3 p2 = mul(Io, w) + cross(h, vin);
    const f3 l2 = mb * vin - cross(h, w);
    const f3 n = mul(Io, al) + cross(h, aa) + cross(w, p2) + cross(vin, l2);
    const f3 f = mb * aa - cross(h, al) + cross(w, l2);
    const float sp = ra.sphi;
    lwb = lwb + sp * n;
    lvb = lvb + sp * f;
    const f3 nb = sp * lw, fb = sp * lv;
    g33 G = {mk(0, 0, 0), mk(0, 0, 0), mk(0, 0, 0)};
    f3 hb = mk(0, 0, 0), p2b = mk(0, 0, 0), l2b = mk(0, 0, 0);
    // n = Io al + h x aa + w x p2 + vin x l2
    g_add_outer(G, nb, al);
    alb = alb + mul(Io, nb);
    hb = hb + cross(aa, nb);
    ab_ = ab_ + cross(nb, h);
    wb_ = wb_ + cross(p2, nb);
    p2b = p2b + cross(nb, w);
    vb_ = vb_ + cross(l2, nb);
    l2b = l2b + cross(nb, vin);
    // f = m aa - h x al + w x l2
    ab_ = ab_ + mb * fb;
    hb = hb - cross(al, fb);
    alb = alb - cross(fb, h);
    wb_ = wb_ + cross(l2, fb);
    l2b = l2b + cross(fb, w);
    // p2 = Io w + h x vin
    g_add_outer(G, p2b, w);
    wb_ = wb_ + mul(Io, p2b);
    hb = hb + cross(vin, p2b);
    vb_ = vb_ + cross(p2b, h);
    // l2 = m vin - h x w
    vb_ = vb_ + mb * l2b;
    hb = hb - cross(w, l2b);
    wb_ = wb_ - cross(l2b, h);
    // body damping: its part of (n, f) is (c_w I_c w + kv r x v_c, kv v_c), I_c = R D R^T,
    // v_c = vin + w x r, kv = c_v m (c_v reduced on a snapped sub-tree); with
    // gv = kv (nb x r + fb) its virtual work is c_w nb . I_c w + gv . v_c
    f3 rdb = mk(0, 0, 0);                               // its cotangent of r
    g33 Gc = {mk(0, 0, 0), mk(0, 0, 0), mk(0, 0, 0)};  // ... and of I_c
    if (a.cv != 0.f || a.cw != 0.f) {
      const float kv = (ws[L.SN + b] != 0.f ? a.cv_snap : a.cv) * mb;
      const f3 vc = vin + cross(w, r);
      const f3 wl = mk(dot(R.c0, w), dot(R.c1, w), dot(R.c2, w));
      const f3 Icw = (Di[0] * wl.x) * R.c0 + (Di[1] * wl.y) * R.c1 + (Di[2] * wl.z) * R.c2;
      lwb = lwb + sp * (a.cw * Icw + kv * cross(r, vc));
      lvb = lvb + (sp * kv) * vc;
      const f3 gv = kv * (cross(nb, r) + fb);
      const f3 nl = mk(dot(R.c0, nb), dot(R.c1, nb), dot(R.c2, nb));
      const f3 Icnb = (Di[0] * nl.x) * R.c0 + (Di[1] * nl.y) * R.c1 + (Di[2] * nl.z) * R.c2;
      vb_ = vb_ + gv;
      wb_ = wb_ + a.cw * Icnb + cross(r, gv);
      rdb = kv * cross(vc, nb) + cross(gv, w);
      g_add_outer(Gc, a.cw * nb, w);
    }
    // Io = R D R^T + m (|r|^2 1 - r r^T), h = m r, r = R com
    const float trG = G.c0.x + G.c1.y + G.c2.z;
    const f3 rb = mb * hb + mb * (2.f * trG * r - g_mulT_plus(G, r)) + rdb;
    Rb_.c0 = Rb_.c0 + com.x * rb + Di[0] * (g_mulT_plus(G, R.c0) + g_mulT_plus(Gc, R.c0));
    Rb_.c1 = Rb_.c1 + com.y * rb + Di[1] * (g_mulT_plus(G, R.c1) + g_mulT_plus(Gc, R.c1));
    Rb_.c2 = Rb_.c2 + com.z * rb + Di[2] * (g_mulT_plus(G, R.c2) + g_mulT_plus(Gc, R.c2));
  }

  // apples hanging from this body
  const int afirst = bi.w & 0x00ffffff, acount = (unsigned)bi.w >> 24;
  for (int k = 0; k < acount; ++k) {
    const int ai = afirst + k, ga = v.a0 + ai;
    const float4 A0 = m.ap0[ga], A1 = m.ap1[ga];
    const f3 hl = xyz(A0);
    const f3 rh = mul(R, hl);
    f3 rhb = mk(0, 0, 0);
    const int det = s.detached[ai];
    if (ra.dyn && det == 0) {
      // the new hang-point velocity seen by the apple update
      const f3 vhb = ld3(wa + A.vh + 3 * ai);
      ovh = ovh + vhb;
      owh = owh + cross(rh, vhb);
      rhb = rhb + cross(vhb, ow);
      // the coupled reaction on the tree (unless on a snapped sub-tree or explicit mode)
      const bool snapped = ws[L.SN + b] != 0.f;
      if (!snapped) {
        const float ma = A0.w, ks = A1.x, csd = A1.y, fdet = A1.z;
        const f3 u = ld3(s.ax + 3 * ai);
        const float D = ma + dt * csd + dt * dt * ks;
        const float beta = dt * dt * ks / D;
        const f3 fr = ks * u - ma * g;
        const f3 avec = ld3(ws + L.AT + 10 * ai);  // the step's a, as recorded
        const float nfr = sqrtf(dot(fr, fr)), fc = a.clamp * fdet;
        const bool clamped = nfr > fc;
        const float sc = clamped ? fc / nfr : 1.f;
        const f3 wv = lv + cross(lw, rh);
        f3 wbar, ubar, vbar;
        if (a.tether_implicit) {
          // psi_a = dt sc [ w.G - dt kap0 w.vh1 ], G = fr + dt k_s avec, kap0 = k_s (1 - beta)
          const f3 G = fr + (dt * ks) * avec;
          const float kap0 = ks * (1.f - beta);
          const f3 vh1 = ov + cross(ow, rh);
          wbar = (dt * sc) * (G - (dt * kap0) * vh1);
          const f3 vh1b = (-dt * dt * sc * kap0) * wv;
          ovb = ovb + vh1b;
          owb = owb + cross(rh, vh1b);
          rhb = rhb + cross(vh1b, ow);
          const float psi_core = dot(wv, G) - dt * kap0 * dot(wv, vh1);
          ubar = (dt * sc * kap0) * wv;
          if (clamped) ubar = ubar + (dt * psi_core * (-sc * ks / (nfr * nfr))) * fr;
          // avec = (ma v + dt (f + ...)) / D; the rails' dependence of f on v is in rails_adjoint
          vbar = (dt * sc * dt * ks * ma / D) * wv;
        } else {
          // psi_a = dt w . (sc fr)
          wbar = (dt * sc) * fr;
          ubar = (dt * sc * ks) * wv;
          if (clamped) ubar = ubar + (dt * dot(wv, fr) * (-sc * ks / (nfr * nfr))) * fr;
          vbar = mk(0, 0, 0);
        }
        lvb = lvb + wbar;
        lwb = lwb + cross(rh, wbar);
        rhb = rhb + cross(wbar, lw);
        float* ub = wa + A.ub + 3 * ai;
        float* vb = wa + A.vb + 3 * ai;
        st3(ub, ld3(ub) + ubar);
        st3(vb, ld3(vb) + vbar);
      }
    }
    if (ra.dyn && det == 2) {
      // converted at this step's start: x = x_hang + u
      const f3 xb_ = ld3(wa + A.ub + 3 * ai);  // cotangent of x (the step-start position)
      xbb = xbb + xb_;
      rhb = rhb + xb_;
    }
    Rb_.c0 = Rb_.c0 + hl.x * rhb;
    Rb_.c1 = Rb_.c1 + hl.y * rhb;
    Rb_.c2 = Rb_.c2 + hl.z * rhb;
  }
  // tips on this body
  if (ra.tipbar) {
    const int tr = m.btip[gb];
    const int tfirst = tr & 0x00ffffff, tcount = (unsigned)tr >> 24;
    for (int k = tfirst; k < tfirst + tcount; ++k) {
      const f3 pb = ld3(ra.tipbar + 3 * (v.t0 + k));
      const f3 tl = xyz(m.tip_local[v.t0 + k]);
      xbb = xbb + pb;
      Rb_.c0 = Rb_.c0 + tl.x * pb;
      Rb_.c1 = Rb_.c1 + tl.y * pb;
      Rb_.c2 = Rb_.c2 + tl.z * pb;
    }
  }

  float c[44];
  cot_put(c, {Rb_, xbb, wb_, vb_, alb, ab_, lwb, lvb, owb, ovb, owh, ovh});
  st_rec(ra.cs + 44 * b, c);
}

HD void reverse_chain(const DevModel& m, const WState& s, const StepArgs& a, const WorldView& v, const AdjLayout& A,
                      float* wa, const RevArgs& ra, int b) {
  const int gb = v.b0 + b;
  const int4 bi = m.bi[gb];
  const int p = bi.x;
  const int dof0 = bi.y & 0x0fffffff, nd = (unsigned)bi.y >> 28;
  const int cfirst = bi.z & 0x00ffffff, ccount = (unsigned)bi.z >> 24;
  const float dt = a.dt;
  // the body's own seeds plus what its children sent
  float cb[44];
  ld_rec(ra.cs + 44 * b, cb);
  for (int k = 0; k < ccount; ++k) {
    float c[44];
    ld_rec(ra.cs + 44 * (cfirst + k), c);
#pragma unroll
    for (int j = 0; j < 44; ++j) cb[j] += c[j];
  }
  const Cot k0 = cot_get(cb);
  m3 Rb_ = k0.R;
  const f3 xbb = k0.x, lvb = k0.lv, ovb = k0.ov, owh = k0.owh, ovh = k0.ovh;
  f3 wb_ = k0.w, vb_ = k0.v, alb = k0.al, ab_ = k0.a, lwb = k0.lw, owb = k0.ow;
  const f3 vin = get3(A.tb + 36 * b, 15);  // the body's own v at x_b

  // reverse of the DOF loop: recompute its intermediates from the parent's tape
  m3 Rp;
  f3 wp, alp, lwp, owp;
  if (p >= 0) {
    float tp[36];
    ld_rec(A.tb + 36 * p, tp);
    Rp = getm(tp, 0);
    wp = get3(tp, 12); alp = get3(tp, 18); lwp = get3(tp, 24); owp = get3(tp, 30);
  } else {
    Rp = {mk(1, 0, 0), mk(0, 1, 0), mk(0, 0, 1)};
    wp = alp = lwp = owp = mk(0, 0, 0);
  }
  const m3 Q = quat_mat(m.bp1[gb]);
  m3 Rs[3];
  f3 ws_[3];
  Rs[0] = mul(Rp, Q);
  ws_[0] = wp;
  float sn_[2], cs_[2];
  for (int j = 0; j < nd; ++j) {
    const int i = dof0 + j;
    const f3 e = j == 0 ? Rs[j].c0 : Rs[j].c1;
    ws_[j + 1] = ws_[j] + s.qd[i] * e;
    sin_cos(s.q[i], &sn_[j], &cs_[j]);
    m3 Rn = Rs[j];
    if (j == 0) {
      Rn.c1 = cs_[j] * Rs[j].c1 + sn_[j] * Rs[j].c2;
      Rn.c2 = cs_[j] * Rs[j].c2 - sn_[j] * Rs[j].c1;
    } else {
      Rn.c0 = cs_[j] * Rs[j].c0 - sn_[j] * Rs[j].c2;
      Rn.c2 = sn_[j] * Rs[j].c0 + cs_[j] * Rs[j].c2;
    }
    Rs[j + 1] = Rn;
  }
  for (int j = nd - 1; j >= 0; --j) {
    const int i = dof0 + j;
    const m3& Rn = Rs[j + 1];
    const m3& Ro = Rs[j];
    // R_new = R_old Rot(q): rotation-angle cotangent and R_old cotangent
    float qbar = 0.f;
    m3 Rob = Rb_;
    if (j == 0) {
      qbar += dot(Rb_.c1, Rn.c2) - dot(Rb_.c2, Rn.c1);
      Rob.c1 = cs_[j] * Rb_.c1 - sn_[j] * Rb_.c2;
      Rob.c2 = sn_[j] * Rb_.c1 + cs_[j] * Rb_.c2;
    } else {
      qbar += -dot(Rb_.c0, Rn.c2) + dot(Rb_.c2, Rn.c0);
      Rob.c0 = cs_[j] * Rb_.c0 + sn_[j] * Rb_.c2;
      Rob.c2 = -sn_[j] * Rb_.c0 + cs_[j] * Rb_.c2;
    }
    Rb_ = Rob;
    const f3 e = j == 0 ? Ro.c0 : Ro.c1;
    const f3 wo = ws_[j];
    const float qd = s.qd[i];
    f3 eb = mk(0, 0, 0);
    float qdbar = 0.f;
    // forward order: alpha += qd (w x e) + qdd e ; a += qd (vin x e) (both with the w before
    // this DOF) ; w += qd e ; Lw += lam e ; Ow += qd1 e. Reversed last to first, so the w
    // update is undone before the alpha term adds its part to w-bar.
    qdbar += dot(wb_, e);
    eb = eb + qd * wb_;
    if (ra.dyn) {
      const float qdd = ra.delta[i] / dt;
      qdbar += dot(alb, cross(wo, e));
      wb_ = wb_ + qd * cross(e, alb);
      eb = eb + qd * cross(alb, wo) + qdd * alb;
      qdbar += dot(ab_, cross(vin, e));
      vb_ = vb_ + qd * cross(e, ab_);
      eb = eb + qd * cross(ab_, vin);
      eb = eb + ra.lam[i] * lwb;
    }
    qdbar += dot(owb, e);  // qd' = qd + Delta with Delta fixed
    eb = eb + ra.qd1[i] * (owb + owh);
    if (j == 0) Rb_.c0 = Rb_.c0 + eb;
    else Rb_.c1 = Rb_.c1 + eb;
    wa[A.qb + i] += qbar;
    wa[A.qdb + i] += qdbar;
  }
  // prefix: R0 = Rp Q, xb = xp + Rp j, d = xb - xp, vin/ain/Lvin/Ovin shifts
  const f3 jb = xyz(m.bp0[gb]);
  const f3 d = mul(Rp, jb);
  f3 db = mk(0, 0, 0);
  // vin = vp + wp x d
  f3 vpb = vb_, wpb = wb_ + cross(d, vb_);
  db = db + cross(vb_, wp);
  // ain = ap + alp x d (a starts at ain; alpha starts at alp)
  f3 apb = ab_, alpb = alb + cross(d, ab_);
  db = db + cross(ab_, alp);
  // Lvin = Lvp + Lwp x d, Ovin = Ovp + Owp x d
  f3 lvpb = lvb, lwpb = lwb + cross(d, lvb);
  db = db + cross(lvb, lwp);
  f3 ovpb = ovb, owpb = owb + cross(d, ovb);
  db = db + cross(ovb, owp);
  f3 ovph = ovh, owph = owh + cross(d, ovh);
  db = db + cross(ovh, owp);
  // d = Rp jb and xb = xp + d
  f3 xpb = xbb;
  db = db + xbb;
  m3 Rpb;
  Rpb.c0 = jb.x * db + (Q.c0.x * Rb_.c0 + Q.c1.x * Rb_.c1 + Q.c2.x * Rb_.c2);
  Rpb.c1 = jb.y * db + (Q.c0.y * Rb_.c0 + Q.c1.y * Rb_.c1 + Q.c2.y * Rb_.c2);
  Rpb.c2 = jb.z * db + (Q.c0.z * Rb_.c0 + Q.c1.z * Rb_.c1 + Q.c2.z * Rb_.c2);
  float c[44];
  cot_put(c, {Rpb, xpb, wpb, vpb, alpb, apb, lwpb, lvpb, owpb, ovpb, owph, ovph});
  st_rec(ra.cs + 44 * b, c);
}

// A solve with the step's factors (see Pivot): L^T sweep leaf to root by factorisation level,
// the scaling z = P^-1 y, and the L sweep root to leaf by body level; y <- H^-1 y, in place.
// With lsweep false it stops after the scaling (the caller does the L sweep, joint by joint).
template <int TPW>
HD void solve_factored(const DevModel& m, const WorldView& v, const WsLayout& L, float* ws, float* y,
                       const Group<TPW>& g, bool lsweep = true) {
  const float* M = ws + L.M;
#ifdef __CUDA_ARCH__
  constexpr int NW = TPW / 32;
  const int warp = g.lane >> 5, lane = g.lane & 31;
  for (int l = v.nBL - 1; l >= 0; --l) {
    const int lo = v.bb[l], hi = v.bb[l + 1];
    if (lo == hi) continue;  // uniform for the group
    if (l > 0) {
      const int count = hi - lo;
      const int2* ft = m.fac_tgt + v.f0 + v.bf[l];
      for (int base = lo; base < hi; base += 32) {
        const int idx = base + lane;
        const bool valid = idx < hi;
        int4 info = make_int4(0, 0, 0, 0);
        float zx = 0.f, zy = 0.f;
        if (valid) {
          info = m.bl_info[v.b0 + idx];
          const Pivot P = pivot_of(M, info.y, info.z, info.w);
          const float yx = y[info.x], yy = (info.w & 3) == 2 ? y[info.x + 1] : 0.f;
          zx = P.p00 * yx + P.p01 * yy;  // P^-1 y of this joint
          zy = P.p01 * yx + P.p11 * yy;
        }
        const bool two = (info.w & 3) == 2;
        const float* rowx = M + info.y;
        const float* rowy = M + (two ? info.z + 1 : info.y);
        const int2* fp = ft + (idx - lo);
        for (int c = 1 + warp; c <= l; c += NW) {
          const int key = valid ? fp[(c - 1) * count].y : -1 - lane;
          const int prev = __shfl_up_sync(0xffffffffu, key, 1);
          const int next = __shfl_down_sync(0xffffffffu, key, 1);
          const bool head = lane == 0 || prev != key;
          const bool tail = lane == 31 || next != key;
          const unsigned heads = __ballot_sync(0xffffffffu, head);
          const int first = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
          const int span = __reduce_max_sync(0xffffffffu, (unsigned)(lane - first + 1));
          const float val = valid ? fmaf(rowx[c], zx, two ? rowy[c] * zy : 0.f) : 0.f;
          const float sum = seg_scan1(val, lane, first, span);
          if (valid && tail) y[key] -= sum;
        }
      }
    }
    g.sync();
    for (int idx = lo + g.lane; idx < hi; idx += TPW) pivot_scale(M, m.bl_info[v.b0 + idx], y);
  }
  g.sync();
#else
  for (int l = v.nBL - 1; l >= 0; --l) {
    const int lo = v.bb[l], hi = v.bb[l + 1];
    const int count = hi - lo;
    const int2* ft = m.fac_tgt + v.f0 + v.bf[l];
    for (int idx = lo; idx < hi; ++idx) {
      const int4 info = m.bl_info[v.b0 + idx];
      const bool two = (info.w & 3) == 2;
      const Pivot P = pivot_of(M, info.y, info.z, info.w);
      const float yx = y[info.x], yy = two ? y[info.x + 1] : 0.f;
      const float zx = P.p00 * yx + P.p01 * yy, zy = P.p01 * yx + P.p11 * yy;
      const float* rowx = M + info.y;
      const float* rowy = M + (two ? info.z + 1 : info.y);
      for (int c = 1; c <= l; ++c) {
        const int2 tk = ft[(c - 1) * count + (idx - lo)];
        y[tk.y] -= fmaf(rowx[c], zx, two ? rowy[c] * zy : 0.f);
      }
    }
    for (int idx = lo; idx < hi; ++idx) pivot_scale(M, m.bl_info[v.b0 + idx], y);
  }
#endif
  if (!lsweep) return;
  // L sweep, root to leaf by body level
  for (int l = 0; l < v.nL; ++l) {
    const int lo = v.lv[l], hi = v.lv[l + 1];
    for (int b = lo + g.lane; b < hi; b += TPW) {
      lsweep_joint(m, v, L, ws, y, m.bi[v.b0 + b].y & 0x0fffffff, m.bj[v.b0 + b]);
    }
    g.sync();
  }
}

// Point loads at the apples' hang points (cotangents vh of the new hang-point velocities):
// adds J_h^T vh to out (per DOF). The moment about a joint origin x_b of its subtree's loads
// is the sum over the subtree's attached apples of (p_a - x_b) x vh_a, p_a the hang point; the
// subtree's apples are one range of apre, so every body sums its own range in a fixed order,
// all bodies at once.
template <int TPW>
HD void hang_load_sweep(const DevModel& m, const WState& s, const WorldView& v, const WsLayout& L,
                        const AdjLayout& A, float* ws, float* wa, float* out, const Group<TPW>& g) {
  for (int b = g.lane; b < v.nb; b += TPW) {
    const int2 r = m.arange[v.b0 + b];
    const int4 bi = m.bi[v.b0 + b];
    const int dof0 = bi.y & 0x0fffffff, nd = (unsigned)bi.y >> 28;
    if (r.x == r.y || nd == 0) continue;
    const f3 xb = ld3(ws + L.X + 3 * b);
    f3 n = mk(0, 0, 0);
    for (int k = r.x; k < r.y; ++k) {
      const int2 ab = m.apre[v.a0 + k];
      if (s.detached[ab.x]) continue;
      const f3 p = ld3(ws + L.X + 3 * ab.y) + ld3(ws + L.AT + 10 * ab.x + 6);
      n = n + cross(p - xb, ld3(wa + A.vh + 3 * ab.x));
    }
    for (int j = 0; j < nd; ++j) out[dof0 + j] += dot(ld3(ws + L.E + 3 * (dof0 + j)), n);
  }
  g.sync();
}

}  // namespace
}  // namespace orchard

namespace orchard {
namespace {

// Springs and dampers of one joint (the diagonal terms of r and H): their part of the q and qd
// cotangents, and the gains' gradients (one writer per joint).
HD void spring_joint(const DevModel& m, const WState& s, const StepArgs& a, const BackArgs& ba, const WorldView& v,
                     const AdjLayout& A, float* wa, int b, int t_abs) {
  const int gb = v.b0 + b;
  const int4 bi = m.bi[gb];
  const int dof0 = bi.y & 0x0fffffff, nd = (unsigned)bi.y >> 28;
  if (nd == 0) return;
  const float dt = a.dt;
  const float4 P3 = m.bp3[gb];
  float k, kd;
  joint_gains(s, a, b, P3, t_abs, &k, &kd);
  const float adt = a.alpha ? dt : 0.f;
  float sk = 0.f, skd = 0.f;
  for (int j = 0; j < nd; ++j) {
    const int i = dof0 + j;
    const float lam = wa[A.lam + i], q1 = wa[A.qd1 + i];
    wa[A.qb + i] += -dt * k * lam;
    wa[A.qdb + i] += -dt * (adt * k + kd) * lam;
    sk += lam * (s.q[i] + adt * q1);
    skd += lam * q1;
  }
  const float kfac = s.broken[b] ? 0.f : 1.f;
  const float kdfac = damper_factor(s, a, b, t_abs);  // d kd' / d kd (also at kd = 0)
  if (ba.dk) ba.dk[gb] += -dt * kfac * sk;
  if (ba.dkd) ba.dkd[gb] += -dt * kdfac * skd;
}

// The rails' part of the cotangent of each apple's start velocity v (App. B: the rails make the
// applied force f a function of v). f enters the apple update, a = (m v + dt (f + m g - k_s u))
// / D when attached and v' = v + dt (g + f / m) when detached, and, through a, the coupled
// reaction on the tree (its virtual work dt sc w . (dt k_s a), w = Lv + Lw x r_h). Both are
// linear in f, so they reach v through one product J^T y of the rails' Jacobian (regimes
// frozen). A pass of its own after the seeds, run only with the rails on, and out of line (its
// code inlined slowed the backward with the rails off).
template <int TPW>
__host__ __device__ __noinline__ void rails_adjoint(const DevModel& m, const WState& s, const StepArgs& a, const WorldView& v, const WsLayout& L,
                      const AdjLayout& A, float* ws, float* wa, const Group<TPW>& g, int t_abs, f3 gv) {
  const float dt = a.dt;
  for (int ai = g.lane; ai < v.na; ai += TPW) {
    const int ga = v.a0 + ai;
    const float4 A0 = m.ap0[ga], A1 = m.ap1[ga];
    const float ma = A0.w, ks = A1.x, csd = A1.y, fdet = A1.z;
    RailTrace rt;
    apply_rails(a, ma, ld3(s.av + 3 * ai), apple_force(a, ga, t_abs), &rt);
    if (!rt.fade && !rt.brake) continue;  // the cap alone does not depend on v
    f3 y = ld3(wa + A.vb1 + 3 * ai) + dt * ld3(wa + A.ub1 + 3 * ai);  // the update's cotangent of v'
    if (s.detached[ai] == 0) {
      const float D = ma + dt * csd + dt * dt * ks;
      y = (dt / D) * y;
      const int b = m.apple_body[ga];
      if (a.tether_implicit && ws[L.SN + b] == 0.f) {
        float t[36];
        ld_rec(A.tb + 36 * b, t);
        const m3 R = getm(t, 0);
        const f3 lw = get3(t, 24), lv = get3(t, 27);
        const f3 rh = mul(R, xyz(A0));
        const f3 fr = ks * ld3(s.ax + 3 * ai) - ma * gv;
        const float nfr = sqrtf(dot(fr, fr)), fc = a.clamp * fdet;
        const float sc = nfr > fc ? fc / nfr : 1.f;
        y = y + (dt * sc * dt * ks * dt / D) * (lv + cross(lw, rh));
      }
    } else {
      y = (dt / ma) * y;
    }
    st3(wa + A.vb + 3 * ai, ld3(wa + A.vb + 3 * ai) + rails_vjp(a, ma, rt, y));
  }
}

// Cotangents of one step (t) of one world: the private state holds the step's start state,
// the forward workspace holds that step's recomputed forward (factors, Delta, apple data), and
// A.qb1 / qdb1 / ub1 / vb1 hold the cotangents of its end state. Leaves the cotangents of its
// start state in A.qb / qdb / ub / vb.
// Phases of the backward for the instrumented build (PhaseClock slots).
enum BackPhase { kBpApples = 0, kBpSolve, kBpLsweep, kBpSeed, kBpChain, kBpRestore, kBpReplay, kBpFinal, kBpOther };

template <int TPW>
HD void reverse_step(const DevModel& m, const WState& s, const StepArgs& a, const BackArgs& ba,
                     const WorldView& v, const WsLayout& L, const AdjLayout& A, float* ws, float* wa, float* cs,
                     const float* kin, const Group<TPW>& g, int t, f3 gv, PhaseClock* pc = nullptr) {
  const float dt = a.dt;
  const int t_abs = a.step0 + t;
  for (int i = g.lane; i < v.nv; i += TPW) {
    wa[A.qb + i] = wa[A.qb1 + i];                                  // q' = q + dt qd'
    wa[A.lam + i] = wa[A.qdb1 + i] + dt * wa[A.qb1 + i];           // qd'-bar (first part)
  }
  // the apple update: u' = u + dt (v' - v_hang'), v' = a + beta v_hang' (attached), or
  // x' = x + dt v', v' = v + dt (g + f / m) (detached); a = (m v + dt (f + m g - k_s u)) / D,
  // f the applied force through the rails (a function of v)
  for (int ai = g.lane; ai < v.na; ai += TPW) {
    const int ga = v.a0 + ai;
    const f3 u1b = ld3(wa + A.ub1 + 3 * ai), v1b = ld3(wa + A.vb1 + 3 * ai);
    const f3 vtot = v1b + dt * u1b;
    if (s.detached[ai] == 0) {
      const float beta = ws[L.AT + 10 * ai + 3];
      const float4 A1 = m.ap1[ga];
      const float ma = m.ap0[ga].w, ks = A1.x, csd = A1.y;
      const float D = ma + dt * csd + dt * dt * ks;
      st3(wa + A.vh + 3 * ai, beta * vtot - dt * u1b);
      st3(wa + A.ub + 3 * ai, u1b - (dt * ks / D) * vtot);
      st3(wa + A.vb + 3 * ai, (ma / D) * vtot);
    } else {
      st3(wa + A.vh + 3 * ai, mk(0, 0, 0));
      st3(wa + A.ub + 3 * ai, u1b);
      st3(wa + A.vb + 3 * ai, vtot);
    }
  }
  g.sync();
  hang_load_sweep<TPW>(m, s, v, L, A, ws, wa, wa + A.lam, g);  // qd'-bar += J_h^T vh-bar
  for (int i = g.lane; i < v.nv; i += TPW) wa[A.qdb + i] = wa[A.lam + i];  // qd' = qd + Delta
  g.sync();
  if (pc) pc->mark(kBpApples);
  solve_factored<TPW>(m, v, L, ws, wa + A.lam, g, false);  // lambda = H^-1 Delta-bar, up to the L sweep
  if (pc) pc->mark(kBpSolve);
  // root to leaf, joint by joint: the L sweep of lambda, the spring and damper terms, and the
  // tape at the step start (which needs the joint's final lambda; kinematics from the record)
  for (int l = 0; l < v.nL; ++l) {
    const int lo = v.lv[l], hi = v.lv[l + 1];
    for (int b = lo + g.lane; b < hi; b += TPW) {
      lsweep_joint(m, v, L, ws, wa + A.lam, m.bi[v.b0 + b].y & 0x0fffffff, m.bj[v.b0 + b]);
      spring_joint(m, s, a, ba, v, A, wa, b, t_abs);
      tape_body_recorded(m, v, L, A, ws, wa, ws + L.r, 1.f / dt, wa + A.lam, wa + A.qd1, b, kin);
    }
    g.sync();
  }
  if (pc) pc->mark(kBpLsweep);
  RevArgs ra;
  ra.dyn = 1;
  ra.delta = ws + L.r;
  ra.lam = wa + A.lam;
  ra.qd1 = wa + A.qd1;
  ra.tipbar = t >= 1 ? ba.dtips + (long long)(t - 1) * a.n_tips_total * 3 : nullptr;
  ra.sphi = -dt;
  ra.cs = cs;
  for (int b = g.lane; b < v.nb; b += TPW) reverse_seed(m, s, a, v, L, A, ws, wa, ra, b, gv, t_abs);
  g.sync();
  if (a.rail_v > 0.f) {
    rails_adjoint<TPW>(m, s, a, v, L, A, ws, wa, g, t_abs, gv);
    g.sync();
  }
  if (pc) pc->mark(kBpSeed);
  for (int l = v.nL - 1; l >= 0; --l) {
    const int lo = v.lv[l], hi = v.lv[l + 1];
    for (int b = lo + g.lane; b < hi; b += TPW) reverse_chain(m, s, a, v, A, wa, ra, b);
    g.sync();
  }
  if (pc) pc->mark(kBpChain);
}

// The seed of the backward pass: the cotangents of the final state from the last record's tips
// (taken at the final configuration, which the staged state holds).
template <int TPW>
HD void reverse_final(const DevModel& m, const WState& s, const StepArgs& a, const BackArgs& ba,
                      const WorldView& v, const WsLayout& L, const AdjLayout& A, float* ws, float* wa, float* cs,
                      const Group<TPW>& g, f3 gv) {
  for (int l = 0; l < v.nL; ++l) {
    const int lo = v.lv[l], hi = v.lv[l + 1];
    for (int b = lo + g.lane; b < hi; b += TPW)
      tape_body(m, s, v, A, wa, wa + A.zero, 0.f, wa + A.zero, wa + A.zero, b, gv);
    g.sync();
  }
  RevArgs ra;
  ra.dyn = 0;
  ra.delta = wa + A.zero; ra.lam = wa + A.zero; ra.qd1 = wa + A.zero;
  ra.tipbar = ba.dtips + (long long)(a.n_steps - 1) * a.n_tips_total * 3;
  ra.sphi = 0.f;
  ra.cs = cs;
  for (int b = g.lane; b < v.nb; b += TPW) reverse_seed(m, s, a, v, L, A, ws, wa, ra, b, gv, a.step0 + a.n_steps);
  g.sync();
  for (int l = v.nL - 1; l >= 0; --l) {
    const int lo = v.lv[l], hi = v.lv[l + 1];
    for (int b = lo + g.lane; b < hi; b += TPW) reverse_chain(m, s, a, v, A, wa, ra, b);
    g.sync();
  }
  for (int i = g.lane; i < v.nv; i += TPW) {
    wa[A.qb1 + i] = wa[A.qb + i];
    wa[A.qb + i] = 0.f;
  }
  g.sync();
}

// The reverse of step t from its start state (snapshot `snap`) and its record `rec`: the
// cotangents of its end state in A.qb1 / qdb1 / ub1 / vb1 become those of its start state.
template <int TPW>
HD void reverse_recorded(const DevModel& m, const WState& s, const StepArgs& a, const BackArgs& ba,
                         const WorldView& v, const WsLayout& L, const AdjLayout& A, float* ws, float* wa, float* cs,
                         const float* snap, const float* rec, const Group<TPW>& g, int t, f3 gv,
                         PhaseClock* pc = nullptr) {
  if (pc) pc->start();
  copy4<TPW>(ws + L.S, snap, A.snap, g);
  const float* kin = rec + WsLayout::kin_offset(v.nb, v.nv, v.nm, v.na);
#ifdef __CUDA_ARCH__
  // the record's kinematics are read level by level in the root-to-leaf sweep: bring them into
  // L2 now, while the rest of the record is copied
  for (int i = g.lane; i < (WsLayout::kKin * v.nb + 31) / 32; i += TPW)
    asm volatile("prefetch.global.L2 [%0];" ::"l"(kin + 32 * i));
#endif
  g.sync();
  step_record<TPW>(ws, L, s, wa, A, v, const_cast<float*>(rec), false, g);
  if (pc) pc->mark(kBpRestore);
  reverse_step<TPW>(m, s, a, ba, v, L, A, ws, wa, cs, kin, g, t, gv, pc);
  for (int i = g.lane; i < v.nv; i += TPW) {
    wa[A.qb1 + i] = wa[A.qb + i];
    wa[A.qdb1 + i] = wa[A.qdb + i];
  }
  for (int i = g.lane; i < 3 * v.na; i += TPW) {
    wa[A.ub1 + i] = wa[A.ub + i];
    wa[A.vb1 + i] = wa[A.vb + i];
  }
  g.sync();
}

// Checkpoint segments over steps [0, t_end), last to first: each is replayed once, forward,
// from its checkpoint, saving every step's start state and record into seg (ckpt_every
// snapshots, then as many records); then its steps are reversed last to first from those.
// seed: the final-tips seed is taken after the last segment's replay (the rollout's end).
template <int TPW>
HD void reverse_segments(const DevModel& m, const StepArgs& a, const BackArgs& ba, const WorldView& v,
                         const WsLayout& L, const AdjLayout& A, const WState& s, float* ws, float* wa, float* cs,
                         float* seg, long long recw, int t_end, bool seed, const Group<TPW>& g, f3 gv,
                         PhaseClock* pc = nullptr) {
  float* recs = seg + (long long)a.ckpt_every * A.snap;
  const int ce = a.ckpt_every;
  const int nseg = (t_end + ce - 1) / ce;
  for (int sg = nseg - 1; sg >= 0; --sg) {
    const int t0 = sg * ce, t1 = (t0 + ce < t_end) ? t0 + ce : t_end;
    if (pc) pc->start();
    load_ckpt(a, v, s, sg, g);
    for (int t = t0; t < t1; ++t) {
      snapshot(ws, L, seg, A, t - t0, true, g);
      float* rec = recs + (long long)(t - t0) * recw;
      step_world<TPW>(m, s, a, v, L, ws, g, a.step0 + t, gv, -1, nullptr,
                      rec + WsLayout::kin_offset(v.nb, v.nv, v.nm, v.na));
      step_record<TPW>(ws, L, s, wa, A, v, rec, true, g);
    }
    if (pc) pc->mark(kBpReplay);
    if (seed && sg == nseg - 1) reverse_final<TPW>(m, s, a, ba, v, L, A, ws, wa, cs, g, gv);
    if (pc) pc->mark(kBpFinal);
    for (int t = t1 - 1; t >= t0; --t)
      reverse_recorded<TPW>(m, s, a, ba, v, L, A, ws, wa, cs, seg + (long long)(t - t0) * A.snap,
                            recs + (long long)(t - t0) * recw, g, t, gv, pc);
  }
}

// Backward pass of one world over a recorded rollout.
// ws: the forward step's temporaries (WsLayout; without a step to replay, MODE 1, the compact
// WsLayout::make_reverse), wa: the backward temporaries (AdjLayout), wt / wc: the tape T / the
// C slots when they are not at wa + A.T / wa + A.C (null: they are), seg: ckpt_every snapshots
// and step records (global memory); ws, wa, wt and wc may be in shared or global memory.
// MODE 0: checkpoints only (reverse_segments over the whole rollout). MODE 1: every step's
// start state and record are in the forward's tape, and the steps are reversed last to first
// straight from it. MODE 2: the tape covers the last a.tape_steps steps, reversed from it
// first; the earlier steps come from their checkpoint segments. The three are separate
// kernels, each compiled for its own path.
template <int TPW, int MODE>
HD void backward_world(const DevModel& m, const StepArgs& a, const BackArgs& ba, int w, float* ws, float* wa,
                       float* wt, float* wc, float* seg, const Group<TPW>& g) {
  const WorldView v = world_view(m, w);
  const WsLayout L = MODE == 1 ? WsLayout::make_reverse(v.nb, v.nv, v.nm, v.na) : WsLayout::make(v.nb, v.nv, v.nm, v.na);
  AdjLayout A = AdjLayout::make(v.nb, v.nv, v.na);
  A.tb = wt ? wt : wa + A.T;
  float* cs = wc ? wc : wa + A.C;
  const WState s = staged_view(ws + L.S, v.nb, v.nv, v.na);  // the world's private state
  const long long recw = WsLayout::record_words(v.nb, v.nv, v.nm, v.na);
  const float4 g4 = m.gravity[w];
  const f3 gv = mk(g4.x, g4.y, g4.z);
  const int T = a.n_steps;
  for (int i = g.lane; i < v.nv; i += TPW) {
    wa[A.qb1 + i] = 0.f; wa[A.qdb1 + i] = 0.f; wa[A.zero + i] = 0.f; wa[A.qb + i] = 0.f; wa[A.qdb + i] = 0.f;
  }
  for (int i = g.lane; i < 3 * v.na; i += TPW) { wa[A.ub1 + i] = 0.f; wa[A.vb1 + i] = 0.f; }
  g.sync();
  PhaseClock* pc = nullptr;
#ifdef ORCHARD_PHASE_CLOCKS
  PhaseClock pcl;
  for (int i = 0; i < kPhaseSlots; ++i) pcl.acc[i] = 0;
  if (a.phase_clk && g.lane == 0) pc = &pcl;
#endif
  if constexpr (MODE == 0) {
    reverse_segments<TPW>(m, a, ba, v, L, A, s, ws, wa, cs, seg, recw, T, true, g, gv, pc);
  } else {
    const int K = a.tape_steps, T1 = T - K;  // the tape holds steps T1 .. T - 1
    const float* tape = a.tape + (long long)(K + 1) * m.tape_off[w];
    const float* trec = tape + (long long)(K + 1) * A.snap;
    copy4<TPW>(ws + L.S, tape + (long long)K * A.snap, A.snap, g);  // the final state
    g.sync();
    if (*s.status & 1u) {
      // the forward froze this world on a non-finite state: its gradients are NaN
      const float nan = u2f(0x7fc00000u);
      for (int i = g.lane; i < v.nb; i += TPW) {
        if (ba.dk) ba.dk[v.b0 + i] += nan;
        if (ba.dkd) ba.dkd[v.b0 + i] += nan;
      }
      for (int i = g.lane; i < v.nv; i += TPW) {
        if (ba.dq0) ba.dq0[v.d0 + i] = nan;
        if (ba.dqd0) ba.dqd0[v.d0 + i] = nan;
      }
      g.sync();
      return;
    }
    if (pc) pc->start();
    reverse_final<TPW>(m, s, a, ba, v, L, A, ws, wa, cs, g, gv);
    if (pc) pc->mark(kBpFinal);
    for (int t = T - 1; t >= T1; --t)
      reverse_recorded<TPW>(m, s, a, ba, v, L, A, ws, wa, cs, tape + (long long)(t - T1) * A.snap,
                            trec + (long long)(t - T1) * recw, g, t, gv, pc);
    if constexpr (MODE == 2)
      reverse_segments<TPW>(m, a, ba, v, L, A, s, ws, wa, cs, seg, recw, T1, false, g, gv, pc);
  }
#ifdef ORCHARD_PHASE_CLOCKS
#ifdef __CUDA_ARCH__
  if (pc) {
    for (int i = 0; i < kPhases; ++i) atomicAdd(a.phase_clk + i, (unsigned long long)pcl.acc[i]);
    atomicAdd(a.phase_clk + kPhases, (unsigned long long)T);  // world-steps reversed
  }
#endif
#endif
  for (int i = g.lane; i < v.nv; i += TPW) {
    if (ba.dq0) ba.dq0[v.d0 + i] = wa[A.qb1 + i];
    if (ba.dqd0) ba.dqd0[v.d0 + i] = wa[A.qdb1 + i];
  }
  g.sync();
}

}  // namespace
}  // namespace orchard
