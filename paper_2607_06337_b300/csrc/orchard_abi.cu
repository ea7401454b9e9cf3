// Host side of liborchard: the C ABI declared in include/orchard.h.
//
// Upload validates a forest descriptor, packs it into FP32 SoA arrays in the caller's device
// buffer, builds the breadth-first level boundaries, the DOF ancestor rows (the storage of the
// tree-sparse mass matrix), the per-world work queue sorted by size class and cost, and the
// default launch schedule of every class. Rollouts launch one persistent kernel per class,
// captured once into a CUDA graph and replayed. No device memory is ever allocated here.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <numeric>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/orchard.h"
#include "orchard_dev.h"

using namespace orchard;

namespace {

std::atomic<int> g_last_cuda{0};
std::atomic<long long> g_launches{0};

ot_status cuda_fail(cudaError_t e) {
  g_last_cuda = (int)e;
  return OT_ECUDA;
}
#define OT_CUDA(call)                           \
  do {                                          \
    cudaError_t e_ = (call);                    \
    if (e_ != cudaSuccess) return cuda_fail(e_); \
  } while (0)

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }
constexpr size_t kSmemLimit = kSmemLimitBytes;  // dynamic shared memory per block (opt-in 227 KB less static)

// Bump allocator over a byte range; in sizing mode it only counts.
struct Carver {
  size_t off = 0;
  template <class T> size_t take(size_t count) {
    size_t o = off;
    off = align_up(off + count * sizeof(T));
    return o;
  }
};

struct ClassInfo {
  int q_begin, q_end;
  int max_nb, max_nv, max_nm, max_na;
  long long ws_floats;
  // the lean placement (WsLayout::make_lean), for classes that fit one world per SM at most:
  // the class's largest shared part and global slot, floats (0: not offered)
  long long lean_ws_floats = 0, lean_slot_floats = 0;
  ot_schedule sched;
  size_t scratch_off;  // byte offset of this class's scratch in the state buffer (global workspace)
  int scratch_slots;
  int back_tpw = 0;    // the backward's threads per world (0: by tree size, see back_plan)
};

// Host-side packed forest (FP32 device layout) plus bookkeeping.
struct Packed {
  int W = 0, NB = 0, NV = 0, NA = 0, NT = 0;
  long long NM = 0;
  std::vector<int> body_off, dof_off, apple_off, tip_off, m_off, lvl_off, lvl;
  std::vector<int4> bi;
  std::vector<float4> bp0, bp1, bp2, bp3, bp4;
  std::vector<int4> bj;               // per body: row starts of its DOFs, first DOF's depth, ndof | fp64
  std::vector<unsigned> anc;
  std::vector<int> bl_off, bl_bound;  // factorisation levels (bodies by first-DOF depth)
  std::vector<int4> bl_info;          // per level position: first DOF, its row, second DOF's row, ndof
  std::vector<int> bl_fbase;          // parallel to bl_bound: each level's start in fac_tgt
  std::vector<int> fac_off;           // [W+1] start of each world's fac_tgt block
  std::vector<int2> fac_tgt;          // per (level, c, position): {row start of the c-th ancestor - c, it}
  std::vector<int> bl_ibase;          // parallel to bl_bound: each level's first work item (world-local)
  std::vector<int> fit_off;           // [W+1] start of each world's work items
  std::vector<int4> fitem;            // factorisation work items {c, first, end position, cost}
  std::vector<float4> ap0, ap1;
  std::vector<int> apple_body, tip_body, btip;
  std::vector<float4> tip_local, gravity;
  std::vector<long long> tape_off;    // [W+1] prefix sums of WsLayout::tape_unit (floats)
  std::vector<int2> apre;             // per apple slot: {apple, its body}, in the bodies' preorder
  std::vector<int2> arange;           // per body: its subtree's slots [x, y) in apre
  std::vector<int> queue;
  std::vector<ClassInfo> classes;
  // domain-randomisation base (empty unless the descriptor has the material): per body
  // {length, diam, rho, E}, {jpos, sigma_r}, {com, armature}; per apple {hang, mass}; per tip
  // the uploaded point
  std::vector<float4> dr_geo, dr_jpos, dr_com, dr_ap0, dr_tip;
};

bool finite_all(const double* p, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(p[i])) return false;
  return true;
}

int num_sms() {
  int dev = 0, n = 148;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 148;
}

ot_schedule default_schedule(long long ws_floats, int max_nb) {
  ot_schedule s{};
  const size_t ws_bytes = (size_t)ws_floats * 4;
  if (ws_bytes > kSmemLimit) {
    s.threads_per_world = 256;
    s.worlds_per_block = 1;
    s.global_workspace = 1;
  } else {
    s.threads_per_world = max_nb <= 96 ? 32 : (max_nb <= 400 ? 64 : 128);
    int g = (int)std::max<size_t>(1, std::min<size_t>(kSmemLimit / std::max<size_t>(ws_bytes, 1), 16));
    if (s.threads_per_world > 32) g = std::min(g, 15);
    g = std::min(g, 512 / s.threads_per_world);
    s.worlds_per_block = std::max(1, std::min(g, s.threads_per_world == 32 ? 4 : 2));
    s.global_workspace = 0;
  }
  s.blocks = 0;
  s.stage = -1;
  return s;
}

ot_status pack(const ot_tree_desc* d, Packed& P, double fp64_twig_diam = 0.0) {
  if (!d || d->n_worlds < 0 || !d->body_off || !d->apple_off || !d->tip_off) return OT_EINVAL;
  const int W = d->n_worlds;
  P.W = W;
  for (int w = 0; w < W; ++w)
    if (d->body_off[w + 1] < d->body_off[w] || d->apple_off[w + 1] < d->apple_off[w] ||
        d->tip_off[w + 1] < d->tip_off[w])
      return OT_EINVAL;
  if (d->body_off[0] != 0 || d->apple_off[0] != 0 || d->tip_off[0] != 0) return OT_EINVAL;
  const int NB = d->body_off[W], NA = d->apple_off[W], NT = d->tip_off[W];
  if (NB > 0 && (!d->parent || !d->ndof || !d->jpos || !d->qrel || !d->com || !d->mass || !d->inertia || !d->k ||
                 !d->kd || !d->armature || !d->m_max))
    return OT_EINVAL;
  if (NA > 0 && (!d->apple_body || !d->hang_local || !d->apple_mass || !d->k_s || !d->c_s || !d->f_detach))
    return OT_EINVAL;
  if (NT > 0 && (!d->tip_body || !d->tip_local)) return OT_EINVAL;
  if (W > 0 && !d->gravity) return OT_EINVAL;
  if (!(fp64_twig_diam >= 0) || !std::isfinite(fp64_twig_diam)) return OT_EINVAL;
  if (fp64_twig_diam > 0 && NB > 0 && !d->diam) return OT_EINVAL;
  // finiteness
  if (NB > 0 && !(finite_all(d->jpos, 3 * (size_t)NB) && finite_all(d->qrel, 4 * (size_t)NB) &&
                  finite_all(d->com, 3 * (size_t)NB) && finite_all(d->mass, NB) &&
                  finite_all(d->inertia, 3 * (size_t)NB) && finite_all(d->k, NB) && finite_all(d->kd, NB) &&
                  finite_all(d->armature, NB) && finite_all(d->m_max, NB)))
    return OT_ENONFINITE;
  if (NA > 0 && !(finite_all(d->hang_local, 3 * (size_t)NA) && finite_all(d->apple_mass, NA) &&
                  finite_all(d->k_s, NA) && finite_all(d->c_s, NA) && finite_all(d->f_detach, NA)))
    return OT_ENONFINITE;
  if (NT > 0 && !finite_all(d->tip_local, 3 * (size_t)NT)) return OT_ENONFINITE;
  if (W > 0 && !finite_all(d->gravity, 3 * (size_t)W)) return OT_ENONFINITE;
  if (fp64_twig_diam > 0 && NB > 0 && !finite_all(d->diam, NB)) return OT_ENONFINITE;
  for (int b = 0; b < NB; ++b)
    if (!(d->mass[b] > 0)) return OT_ENONFINITE;
  for (int a = 0; a < NA; ++a)
    if (!(d->apple_mass[a] > 0)) return OT_ENONFINITE;

  P.body_off.assign(d->body_off, d->body_off + W + 1);
  P.apple_off.assign(d->apple_off, d->apple_off + W + 1);
  P.tip_off.assign(d->tip_off, d->tip_off + W + 1);
  P.dof_off.assign(W + 1, 0);
  P.m_off.assign(W + 1, 0);
  P.lvl_off.assign(W + 1, 0);
  P.bi.resize(NB);
  P.bp0.resize(NB); P.bp1.resize(NB); P.bp2.resize(NB); P.bp3.resize(NB); P.bp4.resize(NB);
  P.bj.assign(NB, make_int4(0, -1, 0, 0));
  P.lvl.clear();
  P.anc.clear();
  P.bl_off.assign(W + 1, 0);
  P.bl_bound.clear();
  P.bl_info.assign(NB, make_int4(0, 0, -1, 0));
  P.bl_fbase.clear();
  P.fac_off.assign(W + 1, 0);
  P.fit_off.assign(W + 1, 0);
  P.bl_ibase.clear();
  P.fitem.clear();
  P.tape_off.assign(W + 1, 0);
  P.apre.assign(NA, make_int2(0, 0));
  P.arange.assign(NB, make_int2(0, 0));
  P.fac_tgt.clear();
  P.btip.clear();
  std::vector<long long> ws(W);
  std::vector<double> cost(W);
  std::vector<int> wnb(W), wnv(W), wnm(W), wna(W);
  int n_dofs = 0;
  for (int w = 0; w < W; ++w) {
    const int b0 = d->body_off[w], nb = d->body_off[w + 1] - b0;
    const int a0 = d->apple_off[w], na = d->apple_off[w + 1] - a0;
    const int t0 = d->tip_off[w], nt = d->tip_off[w + 1] - t0;
    // topology: breadth-first order
    std::vector<int> depth(nb, 0), dof0(nb, 0), nd(nb, 0), cfirst(nb, -1), ccount(nb, 0);
    int nv = 0;
    for (int b = 0; b < nb; ++b) {
      const int p = d->parent[b0 + b];
      const int k = d->ndof[b0 + b];
      if (k < 0 || k > 2) return OT_ETOPO;
      if (b == 0) {
        if (p != -1) return OT_ETOPO;
      } else {
        if (p < 0 || p >= b) return OT_ETOPO;
        if (p < d->parent[b0 + b - 1]) return OT_ETOPO;  // not breadth-first
        depth[b] = depth[p] + 1;
        if (ccount[p] == 0) cfirst[p] = b;
        ++ccount[p];
        if (ccount[p] > 255) return OT_ECAPACITY;
      }
      dof0[b] = nv;
      nd[b] = k;
      nv += k;
    }
    if (nv > 32767 || nb > 65535) return OT_ECAPACITY;
    // apples sorted by body
    std::vector<int> afirst(nb, 0), acount(nb, 0);
    for (int a = 0; a < na; ++a) {
      const int b = d->apple_body[a0 + a];
      if (b < 0 || b >= nb) return OT_ETOPO;
      if (a > 0 && b < d->apple_body[a0 + a - 1]) return OT_ETOPO;
      if (acount[b] == 0) afirst[b] = a;
      if (++acount[b] > 255) return OT_ECAPACITY;
    }
    for (int t = 0; t < nt; ++t) {
      const int b = d->tip_body[t0 + t];
      if (b < 0 || b >= nb) return OT_ETOPO;
      if (t > 0 && b < d->tip_body[t0 + t - 1]) return OT_ETOPO;  // tips sorted by body
    }
    {
      std::vector<int> tf(nb, 0), tc(nb, 0);
      for (int t = 0; t < nt; ++t) {
        const int b = d->tip_body[t0 + t];
        if (tc[b] == 0) tf[b] = t;
        if (++tc[b] > 255) return OT_ECAPACITY;
      }
      for (int b = 0; b < nb; ++b) P.btip.push_back(tf[b] | (tc[b] << 24));
    }
    // levels
    P.lvl_off[w] = (int)P.lvl.size();
    if (nb > 0) {
      P.lvl.push_back(0);
      for (int b = 1; b < nb; ++b)
        if (depth[b] != depth[b - 1]) P.lvl.push_back(b);
      P.lvl.push_back(nb);
    }
    // DOF tree: parent DOF, depth, ancestor rows
    std::vector<int> dpar(nv), ddep(nv), dbody(nv);
    std::vector<int> last_dof(nb, -1);  // deepest DOF on the path root..b
    for (int b = 0; b < nb; ++b) {
      const int p = d->parent[b0 + b];
      int prev = p >= 0 ? last_dof[p] : -1;
      for (int j = 0; j < nd[b]; ++j) {
        const int i = dof0[b] + j;
        dpar[i] = prev;
        ddep[i] = prev >= 0 ? ddep[prev] + 1 : 0;
        if (ddep[i] > kMaxDepth) return OT_ECAPACITY;
        dbody[i] = b;
        prev = i;
      }
      last_dof[b] = prev;
    }
    P.dof_off[w] = n_dofs;
    n_dofs += nv;
    P.m_off[w] = (int)P.anc.size();
    // Ancestor-row storage, laid out by factorisation level (the depth of a joint's first DOF)
    // and, within a level, in its depth-first order: the level's x rows (length l + 1), then
    // its y' rows (length l + 2), each at a stride padded to an odd number of floats. The
    // factorisation reads the rows of 32 consecutive joints of a level at once, one lane each,
    // and an odd stride puts those 32 reads in 32 different shared-memory banks. Every access
    // goes through the row starts (bj, bl_info, fac_tgt, anc), so nothing else depends on it.
    std::vector<int> pre;  // depth-first preorder of the bodies (children in index order)
    {
      pre.reserve(nb);
      std::vector<int> stack;
      if (nb > 0) stack.push_back(0);
      while (!stack.empty()) {
        const int b = stack.back();
        stack.pop_back();
        pre.push_back(b);
        for (int c = ccount[b] - 1; c >= 0; --c) stack.push_back(cfirst[b] + c);
      }
    }
    // apples ordered by their body's preorder position (stable), so that every subtree's
    // apples are one range of slots
    {
      std::vector<int> pos(nb), sub(nb, 1);
      for (int i = 0; i < nb; ++i) pos[pre[i]] = i;
      for (int i = nb - 1; i > 0; --i) sub[d->parent[b0 + pre[i]]] += sub[pre[i]];
      std::vector<int> order(na);
      for (int a = 0; a < na; ++a) order[a] = a;
      std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        return pos[d->apple_body[a0 + x]] < pos[d->apple_body[a0 + y]];
      });
      std::vector<int> key(na);
      for (int k = 0; k < na; ++k) {
        key[k] = pos[d->apple_body[a0 + order[k]]];
        P.apre[a0 + k] = make_int2(order[k], d->apple_body[a0 + order[k]]);
      }
      for (int b = 0; b < nb; ++b) {
        const int lo = (int)(std::lower_bound(key.begin(), key.end(), pos[b]) - key.begin());
        const int hi = (int)(std::lower_bound(key.begin(), key.end(), pos[b] + sub[b]) - key.begin());
        P.arange[b0 + b] = make_int2(lo, hi);
      }
    }
    int maxd = -1;
    for (int b = 0; b < nb; ++b)
      if (nd[b] > 0) maxd = std::max(maxd, ddep[dof0[b]]);
    std::vector<int> rowstart(nv, 0);
    int row = 0;
    for (int l = 0; l <= maxd; ++l) {
      const int sx = (l + 1) | 1, sy = (l + 2) | 1;
      int nx = 0, ny = 0;
      for (int b : pre)
        if (nd[b] > 0 && ddep[dof0[b]] == l) rowstart[dof0[b]] = row + sx * nx++;
      row += sx * nx;
      for (int b : pre)
        if (nd[b] == 2 && ddep[dof0[b]] == l) rowstart[dof0[b] + 1] = row + sy * ny++;
      row += sy * ny;
    }
    const int nm = row;
    {
      std::vector<unsigned> anc_w(nm, 0u);
      for (int i = 0; i < nv; ++i) {
        int j = i;
        for (int c = 0; c <= ddep[i]; ++c) {
          anc_w[rowstart[i] + c] = (unsigned)j | ((unsigned)dbody[j] << 16);
          j = dpar[j];
        }
      }
      P.anc.insert(P.anc.end(), anc_w.begin(), anc_w.end());
    }
    // Factorisation levels: the bodies with DOFs by the depth of their first DOF, each level in
    // depth-first preorder (children in index order), so the bodies of one level below any
    // given DOF are contiguous. Per (level l, ancestor distance c = 1..l, position p): the
    // c-th ancestor of the p-th body's first DOF, as {its row start - c, it}, level-major.
    // The factorisation's work items of a level: for each c, the level's positions split into
    // runs of at most 32 (one warp's chunk) at the boundaries of the groups that share their
    // c-th ancestor (a group larger than 32 stays whole, its chunks in one item), so no two
    // items write the same target row; each level's items sorted by their scan count
    // (chunks x (1 + (l - c + 1) / 8)), largest first, for the warps to take in snake order.
    {
      P.bl_off[w] = (int)P.bl_bound.size();
      P.fac_off[w] = (int)P.fac_tgt.size();
      P.fit_off[w] = (int)P.fitem.size();
      std::vector<int> first;  // first DOF of each level position
      first.reserve(nb);
      int pos = 0, fbase = 0, ibase = 0;
      for (int l = 0; l <= maxd; ++l) {
        P.bl_bound.push_back(pos);
        P.bl_fbase.push_back(fbase);
        P.bl_ibase.push_back(ibase);
        const int lo = pos;
        for (int b : pre)
          if (nd[b] > 0 && ddep[dof0[b]] == l) {
            const int i = dof0[b];
            const bool f64 = fp64_twig_diam > 0 && d->diam[b0 + b] < fp64_twig_diam;
            P.bl_info[b0 + pos] = make_int4(i, rowstart[i], nd[b] == 2 ? rowstart[i + 1] : -1, nd[b] | (f64 ? 16 : 0));
            first.push_back(i);
            ++pos;
          }
        const int count = pos - lo;
        std::vector<int4> items;
        std::vector<int> key(count);
        for (int c = 1; c <= l; ++c) {
          for (int p = 0; p < count; ++p) {
            int j = first[lo + p];
            for (int s2 = 0; s2 < c; ++s2) j = dpar[j];
            P.fac_tgt.push_back(make_int2(rowstart[j] - c, j));
            key[p] = j;
          }
          const int scans = 1 + (l - c + 1) / 8;
          int start = 0, seg = 0;
          for (int p = 1; p <= count; ++p) {
            if (p < count && key[p] == key[p - 1]) continue;  // [seg, p) is one group
            if (p - start > 32 && seg > start) {              // close the run before this group
              items.push_back(make_int4(c, start, seg, ((seg - start + 31) / 32) * scans));
              start = seg;
            }
            if (p - start >= 32) {
              items.push_back(make_int4(c, start, p, ((p - start + 31) / 32) * scans));
              start = p;
            }
            seg = p;
          }
          if (start < count) items.push_back(make_int4(c, start, count, ((count - start + 31) / 32) * scans));
        }
        std::stable_sort(items.begin(), items.end(), [](const int4& a, const int4& b) { return a.w > b.w; });
        P.fitem.insert(P.fitem.end(), items.begin(), items.end());
        fbase += count * l;
        ibase += (int)items.size();
      }
      P.bl_bound.push_back(pos);
      P.bl_fbase.push_back(fbase);
      P.bl_ibase.push_back(ibase);
    }
    for (int b = 0; b < nb; ++b) {
      const int gb = b0 + b;
      if (nd[b] > 0) {
        const int i = dof0[b];
        const bool f64 = fp64_twig_diam > 0 && d->diam[gb] < fp64_twig_diam;
        P.bj[gb] = make_int4(rowstart[i], nd[b] == 2 ? rowstart[i + 1] : -1, ddep[i], nd[b] | (f64 ? 16 : 0));
      }
      if (cfirst[b] < 0) cfirst[b] = 0;
      P.bi[gb] = make_int4(d->parent[gb], dof0[b] | (nd[b] << 28), cfirst[b] | (ccount[b] << 24),
                           afirst[b] | (acount[b] << 24));
      P.bp0[gb] = make_float4((float)d->jpos[3 * gb], (float)d->jpos[3 * gb + 1], (float)d->jpos[3 * gb + 2],
                              (float)d->mass[gb]);
      P.bp1[gb] = make_float4((float)d->qrel[4 * gb], (float)d->qrel[4 * gb + 1], (float)d->qrel[4 * gb + 2],
                              (float)d->qrel[4 * gb + 3]);
      P.bp2[gb] = make_float4((float)d->com[3 * gb], (float)d->com[3 * gb + 1], (float)d->com[3 * gb + 2],
                              (float)d->inertia[3 * gb]);
      P.bp3[gb] = make_float4((float)d->inertia[3 * gb + 1], (float)d->inertia[3 * gb + 2], (float)d->k[gb],
                              (float)d->kd[gb]);
      P.bp4[gb] = make_float4((float)d->armature[gb], (float)d->m_max[gb], 0.f, 0.f);
    }
    wnb[w] = nb; wnv[w] = nv; wnm[w] = nm; wna[w] = na;
    ws[w] = WsLayout::make(nb, nv, nm, na).total;
    P.tape_off[w + 1] = P.tape_off[w] + WsLayout::tape_unit(nb, nv, nm, na);
    long long sumsq = 0;
    for (int i = 0; i < nv; ++i) sumsq += (long long)ddep[i] * (ddep[i] + 1) / 2;
    cost[w] = 700.0 * nb + 12.0 * nm + 2.0 * sumsq + 80.0 * na;
  }
  P.dof_off[W] = n_dofs;
  P.m_off[W] = (int)P.anc.size();
  P.lvl_off[W] = (int)P.lvl.size();
  P.bl_off[W] = (int)P.bl_bound.size();
  P.fac_off[W] = (int)P.fac_tgt.size();
  P.fit_off[W] = (int)P.fitem.size();
  P.NB = NB; P.NA = NA; P.NT = NT; P.NV = P.dof_off[W]; P.NM = P.m_off[W];
  if (P.NM > 0x7fffffffLL) return OT_ECAPACITY;
  // apples, tips, gravity
  P.ap0.resize(NA); P.ap1.resize(NA); P.apple_body.resize(NA);
  for (int a = 0; a < NA; ++a) {
    P.ap0[a] = make_float4((float)d->hang_local[3 * a], (float)d->hang_local[3 * a + 1],
                           (float)d->hang_local[3 * a + 2], (float)d->apple_mass[a]);
    P.ap1[a] = make_float4((float)d->k_s[a], (float)d->c_s[a], (float)d->f_detach[a], 0.f);
    P.apple_body[a] = d->apple_body[a];
  }
  P.tip_body.resize(NT); P.tip_local.resize(NT);
  for (int t = 0; t < NT; ++t) {
    P.tip_body[t] = d->tip_body[t];
    P.tip_local[t] = make_float4((float)d->tip_local[3 * t], (float)d->tip_local[3 * t + 1],
                                 (float)d->tip_local[3 * t + 2], 0.f);
  }
  P.gravity.resize(W);
  for (int w = 0; w < W; ++w)
    P.gravity[w] = make_float4((float)d->gravity[3 * w], (float)d->gravity[3 * w + 1], (float)d->gravity[3 * w + 2], 0.f);
  P.dr_geo.clear(); P.dr_jpos.clear(); P.dr_com.clear(); P.dr_ap0.clear(); P.dr_tip.clear();
  if (d->length && d->rho && d->youngs && d->sigma_r && d->diam) {
    if (!finite_all(d->length, NB) || !finite_all(d->rho, NB) || !finite_all(d->youngs, NB) ||
        !finite_all(d->sigma_r, NB) || !finite_all(d->diam, NB))
      return OT_ENONFINITE;
    for (int b = 0; b < NB; ++b) {
      P.dr_geo.push_back(make_float4((float)d->length[b], (float)d->diam[b], (float)d->rho[b], (float)d->youngs[b]));
      P.dr_jpos.push_back(make_float4((float)d->jpos[3 * b], (float)d->jpos[3 * b + 1], (float)d->jpos[3 * b + 2],
                                      (float)d->sigma_r[b]));
      P.dr_com.push_back(make_float4((float)d->com[3 * b], (float)d->com[3 * b + 1], (float)d->com[3 * b + 2],
                                     (float)d->armature[b]));
    }
    P.dr_ap0 = P.ap0;
    P.dr_tip = P.tip_local;
  }
  // size classes by workspace bytes, queue sorted by (class, cost descending)
  const long long bounds[] = {6 * 1024, 14 * 1024, 28 * 1024, 55 * 1024, (long long)kSmemLimit / 4};
  const int n_bounds = 5;
  // Worlds of one world per SM (above the fourth bound) are split once more: those whose lean
  // placement (WsLayout::make_lean) fits two worlds per SM (228 KB per SM, 1 KB of it reserved
  // per block) form a class of their own, ahead of the rest.
  constexpr long long kLeanPairFloats = (228 * 1024 - 2 * 1024) / 2 / 4;
  std::vector<int> cls(W);
  for (int w = 0; w < W; ++w) {
    int c = 0;
    while (c < n_bounds && ws[w] > bounds[c]) ++c;
    if (c > 3) ++c;
    if (c == 3 && WsLayout::make_lean(wnb[w], wnv[w], (int)wnm[w], wna[w]).total > kLeanPairFloats) c = 4;
    cls[w] = c;
  }
  std::vector<int> order(W);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    if (cls[x] != cls[y]) return cls[x] < cls[y];
    return cost[x] > cost[y];
  });
  P.queue = order;
  P.classes.clear();
  for (int i = 0; i < W;) {
    int j = i;
    ClassInfo ci{};
    ci.q_begin = i;
    while (j < W && cls[order[j]] == cls[order[i]]) {
      const int w = order[j];
      ci.max_nb = std::max(ci.max_nb, wnb[w]);
      ci.max_nv = std::max(ci.max_nv, wnv[w]);
      ci.max_nm = std::max(ci.max_nm, wnm[w]);
      ci.max_na = std::max(ci.max_na, wna[w]);
      ci.ws_floats = std::max(ci.ws_floats, ws[w]);
      ci.lean_ws_floats =
          std::max<long long>(ci.lean_ws_floats, WsLayout::make_lean(wnb[w], wnv[w], (int)wnm[w], wna[w]).total);
      ci.lean_slot_floats = std::max<long long>(ci.lean_slot_floats, WsLayout::lean_slot_floats(wnb[w], wna[w]));
      ++j;
    }
    ci.q_end = j;
    ci.ws_floats = (ci.ws_floats + 3) / 4 * 4;
    ci.sched = default_schedule(ci.ws_floats, ci.max_nb);
    // offered where the whole workspace in shared memory leaves room for one world per SM
    if (ci.sched.global_workspace || (size_t)ci.ws_floats * 4 * 2 <= kSmemLimit) ci.lean_ws_floats = ci.lean_slot_floats = 0;
    P.classes.push_back(ci);
    i = j;
  }
  return OT_OK;
}

template <class T> size_t vbytes(const std::vector<T>& v) { return v.size() * sizeof(T); }

}  // namespace

namespace orchard {
// k and kd live in the z and w lanes of the per-body record bp3.
__global__ void set_gains_kernel(float4* bp3, const float* k, const float* kd, int nb) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  float4 v = bp3[b];
  if (k) v.z = k[b];
  if (kd) v.w = kd[b];
  bp3[b] = v;
}

// Domain randomisation, one block per world (see ot_model_randomize): the world's factors
// (s_len, s_diam, s_rho, s_E, s_sigma, c_d) applied to the uploaded geometry and material, and
// every derived record rebuilt.
struct DrRecords {
  float4 *bp0, *bp2, *bp3, *bp4, *ap0, *tip;
  const float4 *geo, *jpos, *com, *base_ap0, *base_tip;
};
__global__ void dr_build_kernel(DevModel m, DrRecords o, const float* factors, int capsule_links) {
  constexpr float kPi = 3.14159265358979f;
  const int w = blockIdx.x;
  const float* F = factors + 6 * (long long)w;
  const float sl = F[0], sd = F[1], sr = F[2], sE = F[3], ss = F[4], cd = F[5];
  for (int gb = m.body_off[w] + threadIdx.x; gb < m.body_off[w + 1]; gb += blockDim.x) {
    const float4 G = o.geo[gb], J = o.jpos[gb], Cm = o.com[gb];
    const float len = G.x * sl, r = 0.5f * G.y * sd, rho = G.z * sr, E = G.w * sE, sig = J.w * ss;
    const float r2 = r * r;
    float mass, Ixx, Izz;
    if (capsule_links) {  // a cylinder of length len with a hemisphere of radius r on each end
      const float mc = rho * kPi * r2 * len, ms = rho * (4.f / 3.f) * kPi * r2 * r;
      mass = mc + ms;
      Izz = mc * r2 * 0.5f + ms * 0.4f * r2;
      Ixx = mc * (3.f * r2 + len * len) / 12.f + ms * (0.4f * r2 + 0.25f * len * len + 0.375f * len * r);
    } else {              // a solid cylinder
      mass = rho * kPi * r2 * len;
      Izz = mass * r2 * 0.5f;
      Ixx = mass * (3.f * r2 + len * len) / 12.f;
    }
    const bool compliant = ((unsigned)m.bi[gb].y >> 28) > 0;
    const float k = compliant ? kPi * E * r2 * r2 / (4.f * len) : 0.f;
    o.bp0[gb] = make_float4(J.x * sl, J.y * sl, J.z * sl, mass);
    o.bp2[gb] = make_float4(Cm.x * sl, Cm.y * sl, Cm.z * sl, Ixx);
    o.bp3[gb] = make_float4(Ixx, Izz, k, cd * k);
    o.bp4[gb] = make_float4(Cm.w, sig * kPi * r2 * r * 0.25f, 0.f, 0.f);
  }
  for (int ga = m.apple_off[w] + threadIdx.x; ga < m.apple_off[w + 1]; ga += blockDim.x) {
    const float4 H = o.base_ap0[ga];
    o.ap0[ga] = make_float4(H.x * sl, H.y * sl, H.z * sl, H.w);
  }
  for (int gt = m.tip_off[w] + threadIdx.x; gt < m.tip_off[w + 1]; gt += blockDim.x) {
    const float4 T = o.base_tip[gt];
    o.tip[gt] = make_float4(T.x * sl, T.y * sl, T.z * sl, T.w);
  }
}
}  // namespace orchard

struct ot_model {
  Packed P;
  DevModel dev{};
  ot_model_flags flags{};
  int n_sm = 148;
  // the records ot_model_randomize rewrites, and its base (null without the material)
  float4 *w_bp0 = nullptr, *w_bp2 = nullptr, *w_bp3 = nullptr, *w_bp4 = nullptr, *w_ap0 = nullptr,
         *w_tip = nullptr;
  const float4 *dr_geo = nullptr, *dr_jpos = nullptr, *dr_com = nullptr, *dr_ap0 = nullptr, *dr_tip = nullptr;
  unsigned long long* phase_clk = nullptr;  // instrumented builds only: the phase accumulators
  cudaStream_t capture_stream = nullptr;
  struct GraphEntry {
    std::string key;
    cudaGraphExec_t exec = nullptr;
    int kernels = 0;
  };
  std::vector<GraphEntry> graphs;
  // one stream per size class: a captured rollout forks the classes onto them so their launches
  // are independent graph branches that overlap on the GPU
  std::vector<cudaStream_t> class_streams;
  std::vector<cudaEvent_t> join_events;
  cudaEvent_t fork_event = nullptr;
  ~ot_model() {
    for (auto& g : graphs)
      if (g.exec) cudaGraphExecDestroy(g.exec);
    for (cudaStream_t c : class_streams) cudaStreamDestroy(c);
    for (cudaEvent_t e : join_events) cudaEventDestroy(e);
    if (fork_event) cudaEventDestroy(fork_event);
    if (capture_stream) cudaStreamDestroy(capture_stream);
  }
};

struct ot_state {
  const ot_model* model = nullptr;
  DevState dev{};
  int* q_counters = nullptr;  // one per class
  char* base = nullptr;
  size_t bytes = 0;
};

namespace {

// Layout of the packed model in the device buffer.
struct ModelLayout {
  size_t body_off, dof_off, apple_off, tip_off, m_off, lvl_off, lvl, bi, bp0, bp1, bp2, bp3, bp4, bj, anc, bl_off,
      bl_bound, bl_info, bl_fbase, fac_off, fac_tgt, bl_ibase, fit_off, fitem, ap0, ap1, apple_body, tip_body, btip,
      tip_local, gravity, queue,
      dr_geo, dr_jpos, dr_com, dr_ap0, dr_tip, tape_off, apre, arange, total;
};

ModelLayout model_layout(const Packed& P) {
  Carver c;
  ModelLayout L;
  const size_t W1 = P.W + 1;
  L.body_off = c.take<int>(W1); L.dof_off = c.take<int>(W1); L.apple_off = c.take<int>(W1);
  L.tip_off = c.take<int>(W1); L.m_off = c.take<int>(W1); L.lvl_off = c.take<int>(W1);
  L.lvl = c.take<int>(P.lvl.size());
  L.bi = c.take<int4>(P.NB);
  L.bp0 = c.take<float4>(P.NB); L.bp1 = c.take<float4>(P.NB); L.bp2 = c.take<float4>(P.NB);
  L.bp3 = c.take<float4>(P.NB); L.bp4 = c.take<float4>(P.NB);
  L.bj = c.take<int4>(P.NB);
  L.anc = c.take<unsigned>(P.NM);
  L.bl_off = c.take<int>(W1);
  L.bl_bound = c.take<int>(P.bl_bound.size());
  L.bl_info = c.take<int4>(P.bl_info.size());
  L.bl_fbase = c.take<int>(P.bl_fbase.size());
  L.fac_off = c.take<int>(W1);
  L.fac_tgt = c.take<int2>(P.fac_tgt.size());
  L.bl_ibase = c.take<int>(P.bl_ibase.size());
  L.fit_off = c.take<int>(W1);
  L.fitem = c.take<int4>(P.fitem.size());
  L.ap0 = c.take<float4>(P.NA); L.ap1 = c.take<float4>(P.NA);
  L.apple_body = c.take<int>(P.NA);
  L.tip_body = c.take<int>(P.NT);
  L.btip = c.take<int>(P.NB);
  L.tip_local = c.take<float4>(P.NT);
  L.gravity = c.take<float4>(P.W);
  L.queue = c.take<int>(P.W);
  L.dr_geo = c.take<float4>(P.dr_geo.size()); L.dr_jpos = c.take<float4>(P.dr_jpos.size());
  L.dr_com = c.take<float4>(P.dr_com.size()); L.dr_ap0 = c.take<float4>(P.dr_ap0.size());
  L.dr_tip = c.take<float4>(P.dr_tip.size());
  L.tape_off = c.take<long long>(W1);
  L.apre = c.take<int2>(P.NA);
  L.arange = c.take<int2>(P.NB);
  L.total = c.off;
  return L;
}

struct StateLayout {
  size_t q, qd, ax, av, broken, bcnt, break_step, detached, pcnt, tcnt, detach_step, status, counters, total;
  std::vector<size_t> scratch;
};

// Workspace slots of a class in the state's scratch area: classes in shared memory keep one
// (for the plain form); global-workspace classes get four per SM, or one per SM for worlds
// whose temporaries exceed 2 MB.
size_t scratch_slots(const ot_model* m, const ClassInfo& ci) {
  if (ci.sched.global_workspace != 1) return 1;
  return (size_t)m->n_sm * ((size_t)ci.ws_floats * 4 > (2u << 20) ? 1 : 4);
}

// Global slots of a class offered the lean placement: its groups resident at once, at most
// kLeanSlotsPerSm per SM (class_shape caps the launch to them).
constexpr int kLeanSlotsPerSm = 4;
size_t lean_slots(const ot_model* m, const ClassInfo& ci) {
  return ci.lean_slot_floats ? (size_t)kLeanSlotsPerSm * m->n_sm : 0;
}

// A class's scratch (floats): its global-workspace slots, or the lean placement's slots, which
// never run together. Fixed when the model is uploaded, whatever the schedules become.
size_t class_scratch_floats(const ot_model* m, const ClassInfo& ci) {
  return std::max(scratch_slots(m, ci) * (size_t)ci.ws_floats, lean_slots(m, ci) * (size_t)ci.lean_slot_floats);
}

StateLayout state_layout(const ot_model* m) {
  const Packed& P = m->P;
  Carver c;
  StateLayout L;
  L.q = c.take<float>(P.NV); L.qd = c.take<float>(P.NV);
  L.ax = c.take<float>(3 * (size_t)P.NA); L.av = c.take<float>(3 * (size_t)P.NA);
  L.broken = c.take<int>(P.NB); L.bcnt = c.take<int>(P.NB); L.break_step = c.take<int>(P.NB);
  L.detached = c.take<int>(P.NA); L.pcnt = c.take<int>(P.NA); L.tcnt = c.take<int>(P.NA);
  L.detach_step = c.take<int>(P.NA);
  L.status = c.take<unsigned>(P.W);
  L.counters = c.take<int>(std::max<size_t>(P.classes.size(), 1) + 1);
  // scratch: every class may run with global workspace; size for the slots its schedule can
  // have (global classes: 4 blocks of one world per SM; the plain form uses slot 0)
  size_t total_scratch_floats = 0;
  for (const ClassInfo& ci : P.classes) total_scratch_floats += class_scratch_floats(m, ci);
  L.scratch.push_back(c.take<float>(total_scratch_floats));
  L.total = c.off;
  return L;
}

size_t class_scratch_offset(const ot_model* m, int k, int* slots) {
  size_t off = 0;
  for (int i = 0; i < (int)m->P.classes.size(); ++i) {
    const ClassInfo& ci = m->P.classes[i];
    if (i == k) {
      *slots = (int)scratch_slots(m, ci);
      return off;
    }
    off += class_scratch_floats(m, ci);
  }
  *slots = 0;
  return off;
}

long long ckpt_words(const Packed& P) { return 2LL * P.NV + 6LL * P.NA + 3LL * P.NB + 3LL * P.NA; }

StepArgs base_args(const ot_model* m, double dt) {
  StepArgs a{};
  a.dt = (float)dt;
  a.alpha = m->flags.alpha_implicit_spring;
  a.tether_implicit = m->flags.tether_implicit;
  a.n_break = m->flags.n_break;
  a.n_pull = m->flags.n_pull;
  a.n_tension = m->flags.n_tension;
  a.gamma = (float)m->flags.gamma_tension;
  a.clamp = (float)m->flags.clamp_factor;
  a.ramp_inv = m->flags.break_ramp_s > 0 ? (float)(dt / m->flags.break_ramp_s) : 0.f;
  a.ramp_gain = (float)(m->flags.break_ramp_factor - 1.0);
  a.cv = (float)m->flags.lin_damping;
  a.cv_snap = (float)(m->flags.lin_damping * m->flags.snapped_lin_damping);
  a.cw = (float)m->flags.ang_damping;
  if (m->flags.rail_speed > 0) {
    a.rail_v = (float)m->flags.rail_speed;
    a.rail_vf = (float)m->flags.rail_fade_speed;
    a.rail_inv = (float)(1.0 / (m->flags.rail_speed - m->flags.rail_fade_speed));
    a.rail_cap = (float)(m->flags.rail_speed / dt);
    a.rail_cb = (float)m->flags.rail_brake;
  }
  a.single_world = -1;
  a.NB = m->P.NB; a.NV = m->P.NV; a.NA = m->P.NA;
  a.n_tips_total = m->P.NT;
  a.ckpt_words = ckpt_words(m->P);
  return a;
}

// Launch shape of a class under its current schedule (kernel attributes are set here, never
// inside a stream capture).
struct Shape {
  size_t smem;
  int blocks;
  int lean;  // the lean placement (schedule global_workspace 2, allowed for this launch)
  int wpb;   // worlds per block of this launch
  size_t scratch_off;
  int stage_mask;
  long long stage_floats;
  int bps;
};

// Shared-memory floats the staged parts `mask` take for the class's largest world.
long long class_stage_floats(const ot_model* m, const ClassInfo& ci, int mask) {
  const Packed& P = m->P;
  long long mx = 0;
  for (int i = ci.q_begin; i < ci.q_end; ++i) {
    const int w = P.queue[i];
    const StageLayout S = StageLayout::make(mask, P.body_off[w + 1] - P.body_off[w], P.m_off[w + 1] - P.m_off[w],
                                            P.apple_off[w + 1] - P.apple_off[w], P.fac_off[w + 1] - P.fac_off[w],
                                            P.fit_off[w + 1] - P.fit_off[w]);
    mx = std::max<long long>(mx, S.total);
  }
  return mx;
}

// allow_lean false (a rollout that writes the adjoint's tape): a lean schedule runs with its
// whole workspace in shared memory instead.
ot_status class_shape(ot_model* m, int k, Shape* out, bool allow_lean = true) {
  ClassInfo& ci = m->P.classes[k];
  const ot_schedule& sc = ci.sched;
  const bool lean = sc.global_workspace == 2 && allow_lean && ci.lean_slot_floats > 0;
  int wpb = sc.worlds_per_block;
  if (sc.global_workspace == 2 && !lean)  // as many worlds per block as the whole workspace allows
    wpb = (int)std::max<size_t>(1, std::min<size_t>(wpb, kSmemLimit / ((size_t)ci.ws_floats * 4)));
  const size_t ws_block = sc.global_workspace == 1
                              ? 0
                              : (size_t)(lean ? ci.lean_ws_floats : ci.ws_floats) * 4 * wpb;
  if (ws_block > kSmemLimit) return OT_ECAPACITY;
  int bps = 0;
  OT_CUDA(kernel_attributes(sc.threads_per_world, false, lean, wpb, std::max<size_t>(ws_block, 1), &bps));
  if (bps < 1) return OT_ECAPACITY;
  // staged model parts: each part, in kStageOrder, that keeps the blocks per SM of the bare
  // workspace
  int mask = 0;
  long long st = 0;
  if (sc.global_workspace != 1 && sc.stage != 0) {
    if (sc.stage > 0) {
      mask = sc.stage;
      st = class_stage_floats(m, ci, mask);
      if (ws_block + (size_t)st * 4 * wpb > kSmemLimit) return OT_ECAPACITY;
    } else {
      for (int part : kStageOrder) {  // each part that still fits at the same blocks per SM
        const long long st2 = class_stage_floats(m, ci, mask | part);
        const size_t smem2 = ws_block + (size_t)st2 * 4 * wpb;
        if (smem2 > kSmemLimit) continue;
        int bps2 = 0;
        OT_CUDA(kernel_attributes(sc.threads_per_world, true, lean, wpb, smem2, &bps2));
        if (bps2 < bps) continue;
        mask |= part;
        st = st2;
      }
    }
  }
  const size_t smem = ws_block + (size_t)st * 4 * wpb;
  if (mask) OT_CUDA(kernel_attributes(sc.threads_per_world, true, lean, wpb, smem, &bps));
  if (bps < 1) return OT_ECAPACITY;
  out->stage_mask = mask;
  out->stage_floats = st;
  out->bps = bps;
  out->lean = lean ? 1 : 0;
  out->wpb = wpb;
  int slots = 0;
  out->scratch_off = class_scratch_offset(m, k, &slots);
  int blocks = sc.blocks > 0 ? sc.blocks : bps * m->n_sm;
  const int worlds = ci.q_end - ci.q_begin;
  blocks = std::min(blocks, (worlds + wpb - 1) / wpb);
  if (sc.global_workspace == 1) blocks = std::min(blocks, slots / std::max(1, wpb));
  if (lean) blocks = std::min(blocks, (int)(lean_slots(m, ci) / std::max(1, wpb)));
  out->smem = smem;
  out->blocks = blocks;
  return OT_OK;
}

// Launch one class of worlds (persistent, queue-driven) with a precomputed shape.
ot_status launch_class_shaped(ot_model* m, ot_state* s, int k, StepArgs a, const Shape& sh, cudaStream_t st) {
  ClassInfo& ci = m->P.classes[k];
  const ot_schedule& sc = ci.sched;
  if (sh.blocks < 1) return OT_OK;
  a.q_begin = ci.q_begin;
  a.q_end = ci.q_end;
  a.q_counter = s->q_counters + k;
  a.phase_clk = m->phase_clk && k < kBackPhaseRow ? m->phase_clk + (size_t)k * kPhaseSlots : nullptr;
  a.ws_floats = sh.lean ? ci.lean_ws_floats : ci.ws_floats;
  a.global_ws = sc.global_workspace == 1;
  a.lean = sh.lean;
  a.lean_floats = ci.lean_slot_floats;
  a.stage_mask = sh.stage_mask;
  a.stage_floats = sh.stage_floats;
  DevState ds = s->dev;
  ds.scratch = s->dev.scratch + sh.scratch_off;
  OT_CUDA(cudaMemsetAsync(a.q_counter, 0, sizeof(int), st));
  launch_rollout(sc.threads_per_world, sh.wpb, sh.blocks, sh.smem, st, m->dev, ds, a);
  OT_CUDA(cudaGetLastError());
  g_launches += 1;
  return OT_OK;
}

ot_status launch_class(ot_model* m, ot_state* s, int k, StepArgs a, cudaStream_t st) {
  Shape sh;
  ot_status r = class_shape(m, k, &sh);
  if (r != OT_OK) return r;
  return launch_class_shaped(m, s, k, a, sh, st);
}

// One stream and one join event per size class, and the fork event (created once per model):
// the classes of a rollout, a backward or an autotune run concurrently on them.
ot_status ensure_class_streams(ot_model* m) {
  const int nk = (int)m->P.classes.size();
  if (!m->fork_event) OT_CUDA(cudaEventCreateWithFlags(&m->fork_event, cudaEventDisableTiming));
  while ((int)m->class_streams.size() < nk) {
    cudaStream_t c = nullptr;
    cudaEvent_t ev = nullptr;
    OT_CUDA(cudaStreamCreateWithFlags(&c, cudaStreamNonBlocking));
    m->class_streams.push_back(c);
    OT_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    m->join_events.push_back(ev);
  }
  return OT_OK;
}

// Time one launch of every class at its current schedule, the classes concurrent as a rollout
// runs them: each on its own stream, forked from and joined back to st, largest first.
ot_status time_classes_together(ot_model* m, ot_state* s, const StepArgs& a, cudaStream_t st, cudaEvent_t e0,
                                cudaEvent_t e1, float* ms) {
  const int nk = (int)m->P.classes.size();
  OT_CUDA(cudaEventRecord(e0, st));
  OT_CUDA(cudaEventRecord(m->fork_event, st));
  ot_status result = OT_OK;
  for (int k = nk - 1; k >= 0; --k) {
    cudaStream_t sk = m->class_streams[k];
    OT_CUDA(cudaStreamWaitEvent(sk, m->fork_event, 0));
    if (result == OT_OK) result = launch_class(m, s, k, a, sk);
    // always join, so st waits for whatever was enqueued
    OT_CUDA(cudaEventRecord(m->join_events[k], sk));
    OT_CUDA(cudaStreamWaitEvent(st, m->join_events[k], 0));
  }
  OT_CUDA(cudaEventRecord(e1, st));
  if (cudaEventSynchronize(e1) != cudaSuccess) return cuda_fail(cudaGetLastError());
  if (result != OT_OK) return result;
  OT_CUDA(cudaEventElapsedTime(ms, e0, e1));
  return OT_OK;
}

ot_status fill_pulls(StepArgs& a, const ot_force_schedule* pulls) {
  if (pulls && pulls->force) {
    if (!pulls->start || !pulls->end) return OT_EINVAL;
    a.pull_force = pulls->force;
    a.pull_start = pulls->start;
    a.pull_end = pulls->end;
  }
  return OT_OK;
}

}  // namespace

extern "C" {

const char* ot_status_string(ot_status s) {
  switch (s) {
    case OT_OK: return "ok";
    case OT_EINVAL: return "invalid argument";
    case OT_ETOPO: return "bad topology (bodies must be breadth-first, apples sorted by body)";
    case OT_ENONFINITE: return "non-finite or non-positive descriptor value";
    case OT_ECAPACITY: return "world exceeds a hard limit";
    case OT_ECUDA: return "CUDA error";
    case OT_ESTATE: return "call out of order";
    default: return "unknown status";
  }
}

int32_t ot_last_cuda_error(void) { return g_last_cuda.load(); }

int64_t ot_launch_count(int32_t reset) {
  if (reset) return g_launches.exchange(0);
  return g_launches.load();
}

ot_status ot_class_info(ot_model* m, int32_t k, int64_t out[8]) {
  if (!m || !out || k < 0 || k >= (int)m->P.classes.size()) return OT_EINVAL;
  const ClassInfo& ci = m->P.classes[k];
  Shape sh{};
  const ot_status r = class_shape(m, k, &sh);
  if (r != OT_OK) return r;
  out[0] = ci.q_end - ci.q_begin;
  out[1] = ci.max_nb;
  out[2] = (sh.lean ? ci.lean_ws_floats : ci.ws_floats) * 4;
  out[3] = sh.stage_mask;
  out[4] = sh.stage_floats * 4;
  out[5] = (int64_t)sh.smem;
  out[6] = sh.bps;
  out[7] = sh.blocks;
  return OT_OK;
}

ot_status ot_phase_clocks(const ot_model* m, uint64_t* out, int32_t max_classes, int32_t reset) {
  if (!m || !out || max_classes < 1) return OT_EINVAL;
  if (!m->phase_clk) return OT_EINVAL;  // the product build has no phase clocks
  const int nk = std::min<int>(max_classes, kPhaseClasses);
  OT_CUDA(cudaDeviceSynchronize());
  OT_CUDA(cudaMemcpy(out, m->phase_clk, sizeof(uint64_t) * kPhaseSlots * nk, cudaMemcpyDeviceToHost));
  if (reset) OT_CUDA(cudaMemset(m->phase_clk, 0, sizeof(uint64_t) * kPhaseSlots * kPhaseClasses));
  return OT_OK;
}

ot_status ot_model_bytes(const ot_tree_desc* desc, size_t* bytes) {
  if (!bytes) return OT_EINVAL;
  Packed P;
  ot_status st = pack(desc, P);
  if (st != OT_OK) return st;
  *bytes = model_layout(P).total;
  return OT_OK;
}

ot_status ot_tree_model_upload(const ot_tree_desc* desc, const ot_model_flags* flags, void* dev_buf,
                               size_t dev_bytes, void* stream, ot_model** out) {
  if (!out || !dev_buf || !flags) return OT_EINVAL;
  if (((uintptr_t)dev_buf) % kAlign) return OT_EINVAL;
  if (flags->n_break < 1 || flags->n_pull < 1 || flags->n_tension < 1 ||
      (flags->alpha_implicit_spring != 0 && flags->alpha_implicit_spring != 1) ||
      (flags->tether_implicit != 0 && flags->tether_implicit != 1) || !(flags->clamp_factor > 0) ||
      !(flags->gamma_tension > 0) || !(flags->break_ramp_s >= 0) || !(flags->break_ramp_factor >= 0) ||
      !(flags->lin_damping >= 0) || !std::isfinite(flags->lin_damping) || !(flags->ang_damping >= 0) ||
      !std::isfinite(flags->ang_damping) || !(flags->snapped_lin_damping >= 0) ||
      !std::isfinite(flags->snapped_lin_damping) || !(flags->rail_speed >= 0) ||
      !std::isfinite(flags->rail_speed) || !(flags->rail_brake >= 0) || !std::isfinite(flags->rail_brake) ||
      (flags->rail_speed > 0 && !(flags->rail_fade_speed >= 0 && flags->rail_fade_speed < flags->rail_speed)))
    return OT_EINVAL;
  ot_model* m = new ot_model();
  ot_status st = pack(desc, m->P, flags->fp64_twig_diam);
  if (st != OT_OK) {
    delete m;
    return st;
  }
  const Packed& P = m->P;
  ModelLayout L = model_layout(P);
  if (dev_bytes < L.total) {
    delete m;
    return OT_EINVAL;
  }
  m->flags = *flags;
  m->n_sm = num_sms();
  m->phase_clk = phase_clock_buffer();
  std::vector<char> host(L.total, 0);
  auto put = [&](size_t off, const void* src, size_t n) {
    if (n) std::memcpy(host.data() + off, src, n);
  };
  put(L.body_off, P.body_off.data(), vbytes(P.body_off));
  put(L.dof_off, P.dof_off.data(), vbytes(P.dof_off));
  put(L.apple_off, P.apple_off.data(), vbytes(P.apple_off));
  put(L.tip_off, P.tip_off.data(), vbytes(P.tip_off));
  put(L.m_off, P.m_off.data(), vbytes(P.m_off));
  put(L.lvl_off, P.lvl_off.data(), vbytes(P.lvl_off));
  put(L.lvl, P.lvl.data(), vbytes(P.lvl));
  put(L.bi, P.bi.data(), vbytes(P.bi));
  put(L.bp0, P.bp0.data(), vbytes(P.bp0)); put(L.bp1, P.bp1.data(), vbytes(P.bp1));
  put(L.bp2, P.bp2.data(), vbytes(P.bp2)); put(L.bp3, P.bp3.data(), vbytes(P.bp3));
  put(L.bp4, P.bp4.data(), vbytes(P.bp4));
  put(L.bj, P.bj.data(), vbytes(P.bj));
  put(L.anc, P.anc.data(), vbytes(P.anc));
  put(L.bl_off, P.bl_off.data(), vbytes(P.bl_off));
  put(L.bl_bound, P.bl_bound.data(), vbytes(P.bl_bound));
  put(L.bl_info, P.bl_info.data(), vbytes(P.bl_info));
  put(L.bl_fbase, P.bl_fbase.data(), vbytes(P.bl_fbase));
  put(L.fac_off, P.fac_off.data(), vbytes(P.fac_off));
  put(L.fac_tgt, P.fac_tgt.data(), vbytes(P.fac_tgt));
  put(L.bl_ibase, P.bl_ibase.data(), vbytes(P.bl_ibase));
  put(L.fit_off, P.fit_off.data(), vbytes(P.fit_off));
  put(L.fitem, P.fitem.data(), vbytes(P.fitem));
  put(L.ap0, P.ap0.data(), vbytes(P.ap0)); put(L.ap1, P.ap1.data(), vbytes(P.ap1));
  put(L.apple_body, P.apple_body.data(), vbytes(P.apple_body));
  put(L.tip_body, P.tip_body.data(), vbytes(P.tip_body));
  put(L.btip, P.btip.data(), vbytes(P.btip));
  put(L.tip_local, P.tip_local.data(), vbytes(P.tip_local));
  put(L.gravity, P.gravity.data(), vbytes(P.gravity));
  put(L.queue, P.queue.data(), vbytes(P.queue));
  put(L.dr_geo, P.dr_geo.data(), vbytes(P.dr_geo)); put(L.dr_jpos, P.dr_jpos.data(), vbytes(P.dr_jpos));
  put(L.dr_com, P.dr_com.data(), vbytes(P.dr_com)); put(L.dr_ap0, P.dr_ap0.data(), vbytes(P.dr_ap0));
  put(L.dr_tip, P.dr_tip.data(), vbytes(P.dr_tip));
  put(L.tape_off, P.tape_off.data(), vbytes(P.tape_off));
  put(L.apre, P.apre.data(), vbytes(P.apre));
  put(L.arange, P.arange.data(), vbytes(P.arange));
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(dev_buf, host.data(), L.total, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    delete m;
    return cuda_fail(e);
  }
  char* base = (char*)dev_buf;
  DevModel& dm = m->dev;
  dm.W = P.W;
  dm.body_off = (const int*)(base + L.body_off);
  dm.dof_off = (const int*)(base + L.dof_off);
  dm.apple_off = (const int*)(base + L.apple_off);
  dm.tip_off = (const int*)(base + L.tip_off);
  dm.m_off = (const int*)(base + L.m_off);
  dm.lvl_off = (const int*)(base + L.lvl_off);
  dm.lvl = (const int*)(base + L.lvl);
  dm.bi = (const int4*)(base + L.bi);
  dm.bp0 = (const float4*)(base + L.bp0); dm.bp1 = (const float4*)(base + L.bp1);
  dm.bp2 = (const float4*)(base + L.bp2); dm.bp3 = (const float4*)(base + L.bp3);
  dm.bp4 = (const float4*)(base + L.bp4);
  dm.bj = (const int4*)(base + L.bj);
  dm.anc = (const unsigned*)(base + L.anc);
  dm.bl_off = (const int*)(base + L.bl_off);
  dm.bl_bound = (const int*)(base + L.bl_bound);
  dm.bl_info = (const int4*)(base + L.bl_info);
  dm.bl_fbase = (const int*)(base + L.bl_fbase);
  dm.fac_off = (const int*)(base + L.fac_off);
  dm.fac_tgt = (const int2*)(base + L.fac_tgt);
  dm.bl_ibase = (const int*)(base + L.bl_ibase);
  dm.fit_off = (const int*)(base + L.fit_off);
  dm.fitem = (const int4*)(base + L.fitem);
  dm.ap0 = (const float4*)(base + L.ap0); dm.ap1 = (const float4*)(base + L.ap1);
  dm.apple_body = (const int*)(base + L.apple_body);
  dm.tip_body = (const int*)(base + L.tip_body);
  dm.btip = (const int*)(base + L.btip);
  dm.tip_local = (const float4*)(base + L.tip_local);
  dm.gravity = (const float4*)(base + L.gravity);
  dm.queue = (const int*)(base + L.queue);
  dm.tape_off = (const long long*)(base + L.tape_off);
  dm.apre = (const int2*)(base + L.apre);
  dm.arange = (const int2*)(base + L.arange);
  m->w_bp0 = (float4*)(base + L.bp0); m->w_bp2 = (float4*)(base + L.bp2); m->w_bp3 = (float4*)(base + L.bp3);
  m->w_bp4 = (float4*)(base + L.bp4); m->w_ap0 = (float4*)(base + L.ap0); m->w_tip = (float4*)(base + L.tip_local);
  if (!P.dr_geo.empty()) {
    m->dr_geo = (const float4*)(base + L.dr_geo); m->dr_jpos = (const float4*)(base + L.dr_jpos);
    m->dr_com = (const float4*)(base + L.dr_com); m->dr_ap0 = (const float4*)(base + L.dr_ap0);
    m->dr_tip = (const float4*)(base + L.dr_tip);
  }
  *out = m;
  return OT_OK;
}

void ot_model_release(ot_model* model) { delete model; }

ot_status ot_model_set_gains(ot_model* m, const float* k, const float* kd, void* stream) {
  if (!m) return OT_EINVAL;
  if (!k && !kd) return OT_OK;
  const int nb = m->P.NB;
  if (nb == 0) return OT_OK;
  const int threads = 256, blocks = (nb + threads - 1) / threads;
  set_gains_kernel<<<blocks, threads, 0, (cudaStream_t)stream>>>(const_cast<float4*>(m->dev.bp3), k, kd, nb);
  OT_CUDA(cudaGetLastError());
  g_launches += 1;
  return OT_OK;
}

ot_status ot_model_randomize(ot_model* m, const float* factors, int32_t capsule_links, void* stream) {
  if (!m || !factors || !m->dr_geo) return OT_EINVAL;
  if (m->P.W == 0) return OT_OK;
  DrRecords o{m->w_bp0, m->w_bp2, m->w_bp3, m->w_bp4, m->w_ap0, m->w_tip, m->dr_geo, m->dr_jpos, m->dr_com,
              m->dr_ap0, m->dr_tip};
  dr_build_kernel<<<m->P.W, 128, 0, (cudaStream_t)stream>>>(m->dev, o, factors, capsule_links ? 1 : 0);
  OT_CUDA(cudaGetLastError());
  g_launches += 1;
  return OT_OK;
}

ot_status ot_model_counts(const ot_model* m, int64_t counts[6]) {
  if (!m || !counts) return OT_EINVAL;
  counts[0] = m->P.W; counts[1] = m->P.NB; counts[2] = m->P.NV; counts[3] = m->P.NA; counts[4] = m->P.NT;
  counts[5] = (int64_t)m->P.classes.size();
  return OT_OK;
}

ot_status ot_state_bytes(const ot_model* m, size_t* bytes) {
  if (!m || !bytes) return OT_EINVAL;
  *bytes = state_layout(m).total;
  return OT_OK;
}

ot_status ot_world_state_alloc(const ot_model* m, void* dev_buf, size_t bytes, ot_state** out) {
  if (!m || !dev_buf || !out) return OT_EINVAL;
  if (((uintptr_t)dev_buf) % kAlign) return OT_EINVAL;
  StateLayout L = state_layout(m);
  if (bytes < L.total) return OT_EINVAL;
  ot_state* s = new ot_state();
  s->model = m;
  s->base = (char*)dev_buf;
  s->bytes = bytes;
  char* b = s->base;
  s->dev.q = (float*)(b + L.q); s->dev.qd = (float*)(b + L.qd);
  s->dev.ax = (float*)(b + L.ax); s->dev.av = (float*)(b + L.av);
  s->dev.broken = (int*)(b + L.broken); s->dev.bcnt = (int*)(b + L.bcnt); s->dev.break_step = (int*)(b + L.break_step);
  s->dev.detached = (int*)(b + L.detached); s->dev.pcnt = (int*)(b + L.pcnt); s->dev.tcnt = (int*)(b + L.tcnt);
  s->dev.detach_step = (int*)(b + L.detach_step);
  s->dev.status = (unsigned*)(b + L.status);
  s->dev.scratch = (float*)(b + L.scratch[0]);
  s->q_counters = (int*)(b + L.counters);
  *out = s;
  return OT_OK;
}

void ot_state_release(ot_state* s) { delete s; }

ot_status ot_state_set(ot_state* s, const ot_state_init* init, void* stream) {
  if (!s || !init) return OT_EINVAL;
  const Packed& P = s->model->P;
  if (P.NA > 0 && !init->apple_x) return OT_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const cudaMemcpyKind kind = init->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  auto copy_or_zero = [&](void* dst, const void* src, size_t n) -> cudaError_t {
    if (!n) return cudaSuccess;
    if (src) return cudaMemcpyAsync(dst, src, n, kind, st);
    return cudaMemsetAsync(dst, 0, n, st);
  };
  OT_CUDA(copy_or_zero(s->dev.q, init->q, sizeof(float) * P.NV));
  OT_CUDA(copy_or_zero(s->dev.qd, init->qd, sizeof(float) * P.NV));
  OT_CUDA(copy_or_zero(s->dev.ax, init->apple_x, sizeof(float) * 3 * P.NA));
  OT_CUDA(copy_or_zero(s->dev.av, init->apple_v, sizeof(float) * 3 * P.NA));
  const size_t nb = sizeof(int) * P.NB, na = sizeof(int) * P.NA;
  if (nb) {
    OT_CUDA(cudaMemsetAsync(s->dev.broken, 0, nb, st));
    OT_CUDA(cudaMemsetAsync(s->dev.bcnt, 0, nb, st));
    OT_CUDA(cudaMemsetAsync(s->dev.break_step, 0xff, nb, st));
  }
  if (na) {
    OT_CUDA(cudaMemsetAsync(s->dev.detached, 0, na, st));
    OT_CUDA(cudaMemsetAsync(s->dev.pcnt, 0, na, st));
    OT_CUDA(cudaMemsetAsync(s->dev.tcnt, 0, na, st));
    OT_CUDA(cudaMemsetAsync(s->dev.detach_step, 0xff, na, st));
  }
  if (P.W) OT_CUDA(cudaMemsetAsync(s->dev.status, 0, sizeof(unsigned) * P.W, st));
  if (!init->on_device) OT_CUDA(cudaStreamSynchronize(st));
  return OT_OK;
}

ot_status ot_state_get_view(const ot_state* s, ot_state_view* v) {
  if (!s || !v) return OT_EINVAL;
  v->q = s->dev.q; v->qd = s->dev.qd; v->apple_x = s->dev.ax; v->apple_v = s->dev.av;
  v->broken = s->dev.broken; v->break_step = s->dev.break_step;
  v->detached = s->dev.detached; v->detach_step = s->dev.detach_step;
  v->status = s->dev.status;
  return OT_OK;
}

ot_status ot_world_status(const ot_state* s, uint32_t* dev_status, void* stream) {
  if (!s || !dev_status) return OT_EINVAL;
  if (s->model->P.W)
    OT_CUDA(cudaMemcpyAsync(dev_status, s->dev.status, sizeof(unsigned) * s->model->P.W, cudaMemcpyDeviceToDevice,
                            (cudaStream_t)stream));
  return OT_OK;
}

ot_status ot_ckpt_bytes(const ot_model* m, int32_t n_steps, int32_t ckpt_every, size_t* bytes) {
  if (!m || !bytes || n_steps < 0 || ckpt_every < 1) return OT_EINVAL;
  const long long n_snap = (n_steps + ckpt_every - 1) / ckpt_every;
  *bytes = (size_t)(n_snap * ckpt_words(m->P) * 4);
  return OT_OK;
}

ot_status ot_tape_bytes(const ot_model* m, int32_t n_steps, size_t* bytes) {
  if (!m || !bytes || n_steps < 0) return OT_EINVAL;
  *bytes = (size_t)((long long)(n_steps + 1) * m->P.tape_off[m->P.W] * 4);
  return OT_OK;
}

ot_status ot_step(ot_model* m, ot_state* s, const float* ext_force, const ot_force_schedule* pulls, int32_t step,
                  double dt, void* stream) {
  if (!m || !s || s->model != m || !(dt > 0)) return OT_EINVAL;
  StepArgs a = base_args(m, dt);
  a.step0 = step;
  a.n_steps = 1;
  a.ext_force = ext_force;
  ot_status st = fill_pulls(a, pulls);
  if (st != OT_OK) return st;
  for (int k = 0; k < (int)m->P.classes.size(); ++k) {
    st = launch_class(m, s, k, a, (cudaStream_t)stream);
    if (st != OT_OK) return st;
  }
  return OT_OK;
}

ot_status ot_rollout(ot_model* m, ot_state* s, int32_t n_steps, int32_t step0, double dt,
                     const ot_force_schedule* pulls, const ot_record* rec, void* stream) {
  if (!m || !s || s->model != m || n_steps < 0 || !(dt > 0)) return OT_EINVAL;
  if (n_steps == 0) return OT_OK;
  StepArgs a = base_args(m, dt);
  a.step0 = step0;
  a.n_steps = n_steps;
  ot_status st = fill_pulls(a, pulls);
  if (st != OT_OK) return st;
  if (rec) {
    a.tips = rec->tips;
    if (rec->ckpt) {
      if (rec->ckpt_every < 1) return OT_EINVAL;
      size_t need = 0;
      ot_ckpt_bytes(m, n_steps, rec->ckpt_every, &need);
      if (rec->ckpt_bytes < need) return OT_EINVAL;
      a.ckpt = (unsigned*)rec->ckpt;
      a.ckpt_every = rec->ckpt_every;
    }
    if (rec->tape) {
      const int K = rec->tape_steps > 0 ? rec->tape_steps : n_steps;  // the final steps taped
      if (K > n_steps || (K < n_steps && !a.ckpt)) return OT_EINVAL;  // the rest need checkpoints
      size_t need = 0;
      ot_tape_bytes(m, K, &need);
      if (rec->tape_bytes < need || ((uintptr_t)rec->tape) % 16) return OT_EINVAL;
      a.tape = rec->tape;
      a.tape_steps = K;
    }
  }
  cudaStream_t user = (cudaStream_t)stream;
  // graph key: everything the captured launches depend on
  char key[512];
  std::snprintf(key, sizeof(key), "%p|%d|%d|%.17g|%p|%p|%p|%p|%p|%d|%p|%d", (void*)s->base, n_steps, step0, dt,
                (const void*)a.pull_force, (const void*)a.pull_start, (const void*)a.tips, (void*)a.ckpt,
                (const void*)a.pull_end, a.ckpt_every, (void*)a.tape, a.tape_steps);
  std::string skey = key;
  std::string sched_sig;
  for (const ClassInfo& ci : m->P.classes) {
    char b[96];
    std::snprintf(b, sizeof(b), "/%d,%d,%d,%d,%d", ci.sched.threads_per_world, ci.sched.worlds_per_block,
                  ci.sched.blocks, ci.sched.global_workspace, ci.sched.stage);
    sched_sig += b;
  }
  skey += sched_sig;
  for (auto& g : m->graphs)
    if (g.key == skey) {
      OT_CUDA(cudaGraphLaunch(g.exec, user));
      g_launches += g.kernels;
      return OT_OK;
    }
  if (!m->capture_stream) OT_CUDA(cudaStreamCreateWithFlags(&m->capture_stream, cudaStreamNonBlocking));
  cudaStream_t cs = m->capture_stream;
  std::vector<Shape> shapes(m->P.classes.size());
  for (int k = 0; k < (int)m->P.classes.size(); ++k) {
    ot_status r = class_shape(m, k, &shapes[k], a.tape == nullptr);  // no lean placement with a tape
    if (r != OT_OK) return r;
  }
  const int nk = (int)m->P.classes.size();
  {
    const ot_status r = ensure_class_streams(m);
    if (r != OT_OK) return r;
  }
  OT_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  const long long before = g_launches.load();
  ot_status rst = OT_OK;
  cudaError_t ce = cudaEventRecord(m->fork_event, cs);
  // largest classes first: they hold the longest-running worlds
  int forked = 0;
  for (int k = nk - 1; k >= 0 && ce == cudaSuccess; --k) {
    cudaStream_t sk = m->class_streams[k];
    ce = cudaStreamWaitEvent(sk, m->fork_event, 0);
    if (ce != cudaSuccess) break;
    ++forked;
    if (rst == OT_OK) rst = launch_class_shaped(m, s, k, a, shapes[k], sk);
    ce = cudaEventRecord(m->join_events[k], sk);
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(cs, m->join_events[k], 0);
  }
  (void)forked;
  if (ce != cudaSuccess && rst == OT_OK) rst = cuda_fail(ce);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(cs, &graph);
  const int kernels = (int)(g_launches.load() - before);
  g_launches -= kernels;  // capture is not execution
  if (rst != OT_OK) {
    if (graph) cudaGraphDestroy(graph);
    return rst;
  }
  if (e != cudaSuccess) return cuda_fail(e);
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(e);
  if (m->graphs.size() >= 8) {
    cudaGraphExecDestroy(m->graphs.front().exec);
    m->graphs.erase(m->graphs.begin());
  }
  m->graphs.push_back({skey, exec, kernels});
  OT_CUDA(cudaGraphLaunch(exec, user));
  g_launches += kernels;
  return OT_OK;
}

ot_status ot_rollout_plain(ot_model* m, ot_state* s, int32_t n_steps, int32_t step0, double dt,
                           const ot_force_schedule* pulls, void* stream) {
  if (!m || !s || s->model != m || n_steps < 0 || !(dt > 0)) return OT_EINVAL;
  StepArgs a = base_args(m, dt);
  ot_status st = fill_pulls(a, pulls);
  if (st != OT_OK) return st;
  a.n_steps = 1;
  cudaStream_t cs = (cudaStream_t)stream;
  // one fixed launch shape for every world: 64 threads, workspace in shared memory when it
  // fits, else in the first scratch slot of the world's class
  const Packed& P = m->P;
  std::vector<int> cls_of(P.W);
  for (int k = 0; k < (int)P.classes.size(); ++k)
    for (int i = P.classes[k].q_begin; i < P.classes[k].q_end; ++i) cls_of[P.queue[i]] = k;
  // the largest shared-memory size any world needs, set once
  size_t smem_max = 1;
  for (const ClassInfo& ci : P.classes)
    if ((size_t)ci.ws_floats * 4 <= kSmemLimit) smem_max = std::max(smem_max, (size_t)ci.ws_floats * 4);
  int bps = 0;
  OT_CUDA(kernel_attributes(64, false, false, 1, smem_max, &bps));
  for (int t = 0; t < n_steps; ++t) {
    a.step0 = step0 + t;
    for (int w = 0; w < P.W; ++w) {
      const ClassInfo& ci = P.classes[cls_of[w]];
      StepArgs b = a;
      b.single_world = w;
      b.ws_floats = ci.ws_floats;
      const bool fits = (size_t)ci.ws_floats * 4 <= kSmemLimit;
      b.global_ws = fits ? 0 : 1;
      DevState ds = s->dev;
      int slots = 0;
      ds.scratch = s->dev.scratch + class_scratch_offset(m, cls_of[w], &slots);
      const size_t smem = fits ? (size_t)ci.ws_floats * 4 : 0;
      launch_rollout(64, 1, 1, smem, cs, m->dev, ds, b);
      OT_CUDA(cudaGetLastError());
      g_launches += 1;
    }
  }
  return OT_OK;
}

ot_status ot_get_schedule(const ot_model* m, int32_t k, ot_schedule* sc) {
  if (!m || !sc || k < 0 || k >= (int)m->P.classes.size()) return OT_EINVAL;
  *sc = m->P.classes[k].sched;
  return OT_OK;
}

ot_status ot_set_schedule(ot_model* m, int32_t k, const ot_schedule* sc) {
  if (!m || !sc || k < 0 || k >= (int)m->P.classes.size()) return OT_EINVAL;
  const ClassInfo& ci = m->P.classes[k];
  const int t = sc->threads_per_world;
  if (t != 32 && t != 64 && t != 128 && t != 256 && t != 512) return OT_EINVAL;
  if (sc->worlds_per_block < 1 || t * sc->worlds_per_block > 512) return OT_EINVAL;
  if (t > 32 && sc->worlds_per_block > 15) return OT_EINVAL;
  if (t == 32 && sc->worlds_per_block > 16) return OT_EINVAL;
  if (sc->blocks < 0) return OT_EINVAL;
  // a class's global-workspace setting (1) is fixed at upload (it sizes the state's scratch);
  // a class in shared memory may take the lean placement (2) where it is offered
  const int gw = sc->global_workspace;
  if (gw < 0 || gw > 2) return OT_EINVAL;
  if ((gw == 1) != (ci.sched.global_workspace == 1)) return OT_EINVAL;
  if (gw == 2 && (!ci.lean_slot_floats || t < 128)) return OT_EINVAL;  // instantiated for 128-512 threads
  if (gw == 0 && (size_t)ci.ws_floats * 4 * sc->worlds_per_block > kSmemLimit) return OT_EINVAL;
  if (gw == 2 && ((size_t)ci.lean_ws_floats * 4 * sc->worlds_per_block > kSmemLimit ||
                  (size_t)sc->worlds_per_block * std::max(sc->blocks, 1) > lean_slots(m, ci)))
    return OT_EINVAL;
  if (gw == 1 && (size_t)sc->worlds_per_block * std::max(sc->blocks, 1) > scratch_slots(m, ci))
    return OT_EINVAL;
  if (sc->stage < -1 || sc->stage > 127) return OT_EINVAL;
  m->P.classes[k].sched = *sc;
  return OT_OK;
}

ot_status ot_autotune(ot_model* m, ot_state* s, int32_t n_steps, double dt, void* stream) {
  if (!m || !s || s->model != m || n_steps < 1 || !(dt > 0)) return OT_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  {
    const ot_status r = ensure_class_streams(m);
    if (r != OT_OK) return r;
  }
  // Every timed launch starts from the state as it was at the call (the state arrays, q to the
  // status words, are contiguous from the buffer's base): a candidate timed on a state that
  // earlier candidates have advanced would not be timed on the same work. Restored at the end.
  const size_t state_bytes = state_layout(m).counters;
  void* saved = nullptr;
  OT_CUDA(cudaMalloc(&saved, std::max<size_t>(state_bytes, 16)));
  OT_CUDA(cudaMemcpyAsync(saved, s->base, state_bytes, cudaMemcpyDeviceToDevice, st));
  auto restore = [&]() { return cudaMemcpyAsync(s->base, saved, state_bytes, cudaMemcpyDeviceToDevice, st); };
  cudaEvent_t e0, e1;
  OT_CUDA(cudaEventCreate(&e0));
  OT_CUDA(cudaEventCreate(&e1));
  StepArgs a = base_args(m, dt);
  a.n_steps = n_steps;
  ot_status result = OT_OK;
  const int nk = (int)m->P.classes.size();
  // Pass 1, each class alone: every candidate timed once after a warm-up; the fastest few kept.
  constexpr int kKeep = 3;
  std::vector<std::vector<ot_schedule>> kept(nk);
  for (int k = 0; k < nk && result == OT_OK; ++k) {
    ClassInfo& ci = m->P.classes[k];
    const ot_schedule keep = ci.sched;
    std::vector<ot_schedule> cands;
    // placements: the class's own (all in global memory, or all in shared memory), and the lean
    // one where it is offered
    const int base_gw = keep.global_workspace == 1 ? 1 : 0;
    for (int gw : {base_gw, 2}) {
      if (gw == 2 && (base_gw == 1 || !ci.lean_slot_floats)) continue;
      const long long wsf = gw == 2 ? ci.lean_ws_floats : ci.ws_floats;
      for (int t : {32, 64, 128, 256, 512})
        for (int g : {1, 2, 3, 4, 6, 8, 12, 16})
          for (int stage : {0, -1}) {  // model records read from global memory, or staged
            ot_schedule c{t, g, 0, gw, stage};
            if (t * g > 512) continue;
            if (t > 32 && g > 15) continue;
            if (gw != 1 && (size_t)wsf * 4 * g > kSmemLimit) continue;
            if (gw == 1 && (g > 1 || stage != 0)) continue;
            if (gw == 2 && ((size_t)g > lean_slots(m, ci) || t < 128)) continue;
            cands.push_back(c);
          }
    }
    std::vector<std::pair<float, int>> timed;
    for (int i = 0; i < (int)cands.size(); ++i) {
      const ot_schedule& c = cands[i];
      ci.sched = c;
      if (c.stage == -1) {  // automatic staging that stages nothing repeats the stage-0 candidate
        Shape sh{};
        if (class_shape(m, k, &sh) != OT_OK || sh.stage_mask == 0) continue;
      }
      float ms = 0;
      ot_status r = launch_class(m, s, k, a, st);  // warm-up and attribute set-up
      if (r != OT_OK) continue;
      if (restore() != cudaSuccess) {
        result = cuda_fail(cudaGetLastError());
        break;
      }
      cudaEventRecord(e0, st);
      r = launch_class(m, s, k, a, st);
      cudaEventRecord(e1, st);
      if (r != OT_OK) continue;
      if (cudaEventSynchronize(e1) != cudaSuccess) {
        result = cuda_fail(cudaGetLastError());
        break;
      }
      cudaEventElapsedTime(&ms, e0, e1);
      timed.push_back({ms, i});
    }
    std::sort(timed.begin(), timed.end());
    for (int j = 0; j < (int)timed.size() && j < kKeep; ++j) kept[k].push_back(cands[timed[j].second]);
    ci.sched = kept[k].empty() ? keep : kept[k][0];
  }
  // Pass 2, the classes together as a rollout runs them (concurrently, one stream each): a
  // schedule that is fastest alone can lose once the other classes share the SMs. Largest class
  // first, each kept candidate is timed with the others at their current choice (best of two
  // timings after a warm-up), and the one with the shortest whole-batch time stays. With one
  // class this re-times its kept candidates, best of two, against the noise of a single timing.
  for (int k = nk - 1; k >= 0 && result == OT_OK; --k) {
    ClassInfo& ci = m->P.classes[k];
    if (kept[k].size() < 2) continue;
    float best = 1e30f;
    ot_schedule best_s = ci.sched;
    for (const ot_schedule& c : kept[k]) {
      ci.sched = c;
      float ms = 1e30f;
      for (int rep = 0; rep < 3 && result == OT_OK; ++rep) {
        float t = 0;
        if (restore() != cudaSuccess) {
          result = cuda_fail(cudaGetLastError());
          break;
        }
        const ot_status r = time_classes_together(m, s, a, st, e0, e1, &t);
        if (r == OT_ECUDA) result = r;
        if (r != OT_OK) break;
        if (rep > 0) ms = std::min(ms, t);  // the first launch is the warm-up
      }
      if (ms < best) {
        best = ms;
        best_s = c;
      }
    }
    ci.sched = best_s;
  }
  if (restore() != cudaSuccess && result == OT_OK) result = cuda_fail(cudaGetLastError());
  if (cudaStreamSynchronize(st) != cudaSuccess && result == OT_OK) result = cuda_fail(cudaGetLastError());
  cudaFree(saved);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return result;
}

namespace {
// Backward launch plan of a class: threads per world by the class's largest tree;
// the forward step's temporaries in shared memory when they fit, the backward's and the
// segment snapshots in global memory; one workspace slot per group that can be resident at
// once (bounded by shared memory, registers and 16 groups per SM).
struct BackPlan {
  int tpw, gpb, blocks;
  size_t slots;
  BackShape sh;
};
inline long long round16(long long f) { return (f + 15) / 16 * 16; }

constexpr int kBackTpw[3] = {64, 128, 256};  // the backward's candidate threads per world

BackPlan back_plan(const ot_model* m, const ClassInfo& ci, int ce, int tpw = 0) {
  BackPlan p{};
  // threads per world: as given, as the class's backward schedule says, or by tree size
  // (measured on B300 with 200-body trees: 256 beat 128)
  p.tpw = tpw > 0 ? tpw : ci.back_tpw > 0 ? ci.back_tpw : (ci.max_nb <= 96 ? 64 : 256);
  BackShape& sh = p.sh;
  // without checkpoints no step is replayed: the reverse needs only the compact forward layout
  sh.fwd_floats = round16(ce == 0 ? backward_reverse_ws_floats(ci.max_nb, ci.max_nv, ci.max_nm, ci.max_na)
                                  : ci.ws_floats);
  sh.adj_floats = round16(backward_adj_floats(ci.max_nb, ci.max_nv, ci.max_na));
  sh.small_floats = round16(backward_adj_small_floats(ci.max_nb, ci.max_nv, ci.max_na));
  sh.head_floats = round16(backward_adj_head_floats(ci.max_nb, ci.max_nv, ci.max_na));
  sh.t_floats = round16(36LL * ci.max_nb);
  sh.c_floats = round16(44LL * ci.max_nb);
  const long long seg = round16(backward_seg_floats(ci.max_nb, ci.max_nv, ci.max_nm, ci.max_na, ce));
  const long long lim = (long long)(kSmemLimit / 4);
  // resident groups per SM the registers allow (the kernel is built for 128 per thread)
  const long long by_regs = std::min<long long>(std::min<long long>(2048, 65536 / 128) / p.tpw, 16);
  // The placement with the most groups resident per SM, then the most in shared memory
  // (measured on B300 with diff1024 trees: more resident worlds beat more shared memory per
  // world, and at equal residency the backward's temporaries in shared memory beat global).
  struct Placement {
    int mode;
    long long smem, global;
  };
  const Placement cand[5] = {{2, sh.fwd_floats + sh.adj_floats, seg},
                             {3, sh.fwd_floats + sh.head_floats, sh.c_floats + seg},
                             {4, sh.fwd_floats + sh.small_floats, sh.t_floats + sh.c_floats + seg},
                             {1, sh.fwd_floats, sh.adj_floats + seg},
                             {0, 0, sh.fwd_floats + sh.adj_floats + seg}};
  long long best = -1;
  for (const Placement& c : cand) {
    if (c.smem > lim) continue;
    const long long per = c.smem > 0 ? std::min(by_regs, lim / c.smem) : by_regs;
    if (per > best) {
      best = per;
      sh.mode = c.mode;
      sh.smem_floats = c.smem;
      sh.global_floats = c.global;
    }
  }
  sh.global_floats = (sh.global_floats + 63) / 64 * 64;
  // groups per block: as many as share one block's shared memory (at most kBackMaxThreads threads)
  p.gpb = sh.smem_floats > 0
              ? (int)std::max<long long>(1, std::min<long long>(lim / sh.smem_floats, kBackMaxThreads / p.tpw))
              : 1;
  p.gpb = std::min(p.gpb, 16);
  // resident groups per SM
  long long per_sm = by_regs;
  if (sh.smem_floats > 0) per_sm = std::min<long long>(per_sm, (long long)(kSmemLimit / 4) / sh.smem_floats);
  per_sm = std::max<long long>(per_sm, 1);
  const size_t worlds = (size_t)(ci.q_end - ci.q_begin);
  p.slots = std::min<size_t>(worlds, (size_t)m->n_sm * (size_t)per_sm);
  p.slots = (p.slots + p.gpb - 1) / p.gpb * p.gpb;
  p.blocks = (int)(p.slots / p.gpb);
  return p;
}
// A class's share of the backward workspace (floats): enough for any of the candidate threads
// per world, so that the layout does not depend on the class's backward schedule.
size_t back_class_floats(const ot_model* m, const ClassInfo& ci, int ce) {
  size_t mx = 0;
  for (int t : kBackTpw) {
    const BackPlan p = back_plan(m, ci, ce, t);
    mx = std::max(mx, p.slots * (size_t)p.sh.global_floats);
  }
  return mx;
}

// The backward's arguments from ot_rollout_backward's (validated; see orchard.h).
ot_status backward_args(ot_model* m, ot_state* s, int32_t n_steps, int32_t step0, double dt,
                        const ot_force_schedule* pulls, const ot_record* rec, const float* dL_dtips, ot_grads* grads,
                        void* workspace, size_t workspace_bytes, StepArgs* out, BackArgs* ba, int* ce_out) {
  if (!m || !s || s->model != m || n_steps < 1 || !(dt > 0) || !rec || !dL_dtips || !grads) return OT_EINVAL;
  // the tape when the forward wrote one; checkpoints (and segment replays) for the steps before
  // a tape of the final steps only, or for all steps without a tape
  const bool tape = rec->tape != nullptr;
  const int K = tape ? (rec->tape_steps > 0 ? rec->tape_steps : n_steps) : 0;
  if (K > n_steps) return OT_EINVAL;
  const bool need_ckpt = K < n_steps;
  if (need_ckpt && (!rec->ckpt || rec->ckpt_every < 1)) return OT_ESTATE;
  if (((uintptr_t)workspace) % kAlign) return OT_EINVAL;
  const int ce = need_ckpt ? rec->ckpt_every : 0;
  size_t need = 0;
  if (tape) {
    ot_tape_bytes(m, K, &need);
    if (rec->tape_bytes < need || ((uintptr_t)rec->tape) % 16) return OT_EINVAL;
  }
  if (need_ckpt) {
    ot_ckpt_bytes(m, n_steps, ce, &need);
    if (rec->ckpt_bytes < need) return OT_EINVAL;
  }
  ot_backward_workspace_bytes(m, ce, &need);
  if (workspace_bytes < need || (need > 0 && !workspace)) return OT_EINVAL;  // none needed: may be null
  StepArgs a = base_args(m, dt);
  a.step0 = step0;
  a.n_steps = n_steps;
  ot_status st = fill_pulls(a, pulls);
  if (st != OT_OK) return st;
  if (tape) {
    a.tape = rec->tape;
    a.tape_steps = K;
  }
  if (need_ckpt) {
    a.ckpt = (unsigned*)rec->ckpt;
    a.ckpt_every = ce;
  }
  *out = a;
  *ba = BackArgs{dL_dtips, grads->dk, grads->dkd, grads->dq0, grads->dqd0};
  *ce_out = ce;
  return OT_OK;
}

// The start of class k's share of the backward workspace.
float* back_work(const ot_model* m, float* work, int k, int ce) {
  for (int i = 0; i < k; ++i) work += back_class_floats(m, m->P.classes[i], ce);
  return work;
}

// Launch class k's backward on stream sk with its current plan.
cudaError_t launch_back_class(ot_model* m, ot_state* s, int k, const StepArgs& a, const BackArgs& ba, float* work,
                              int ce, cudaStream_t sk) {
  const ClassInfo& ci = m->P.classes[k];
  const BackPlan p = back_plan(m, ci, ce);
  int bps = 0;
  const int mode = !a.tape ? 0 : a.tape_steps < a.n_steps ? 2 : 1;
  cudaError_t e = backward_attributes(p.tpw, mode, p.gpb, (size_t)p.sh.smem_floats * 4 * p.gpb, &bps);
  if (e == cudaSuccess && bps < 1) e = cudaErrorInvalidConfiguration;
  StepArgs b = a;
  b.q_begin = ci.q_begin;
  b.q_end = ci.q_end;
  b.q_counter = s->q_counters + k;
  // instrumented builds: the backward's phase clocks of class k sit in row kBackPhaseRow + k
  b.phase_clk = m->phase_clk && k < kPhaseClasses - kBackPhaseRow
                    ? m->phase_clk + (size_t)(kBackPhaseRow + k) * kPhaseSlots : nullptr;
  if (e == cudaSuccess) e = cudaMemsetAsync(b.q_counter, 0, sizeof(int), sk);
  if (e == cudaSuccess && p.blocks > 0) {
    launch_backward(p.tpw, p.gpb, p.blocks, sk, m->dev, b, ba, work, p.sh);
    e = cudaGetLastError();
    if (e == cudaSuccess) g_launches += 1;
  }
  return e;
}
}  // namespace

ot_status ot_backward_workspace_bytes(const ot_model* m, int32_t ckpt_every, size_t* bytes) {
  if (!m || !bytes || ckpt_every < 0) return OT_EINVAL;
  size_t total = 0;
  for (const ClassInfo& ci : m->P.classes) total += back_class_floats(m, ci, ckpt_every) * 4;
  *bytes = total;
  return OT_OK;
}

ot_status ot_get_backward_schedule(const ot_model* m, int32_t k, int32_t* threads_per_world) {
  if (!m || !threads_per_world || k < 0 || k >= (int)m->P.classes.size()) return OT_EINVAL;
  *threads_per_world = back_plan(m, m->P.classes[k], 0).tpw;
  return OT_OK;
}

ot_status ot_set_backward_schedule(ot_model* m, int32_t k, int32_t threads_per_world) {
  if (!m || k < 0 || k >= (int)m->P.classes.size()) return OT_EINVAL;
  const int t = threads_per_world;
  if (t != 0 && t != 64 && t != 128 && t != 256) return OT_EINVAL;
  m->P.classes[k].back_tpw = t;
  return OT_OK;
}

ot_status ot_autotune_backward(ot_model* m, ot_state* s, int32_t n_steps, int32_t step0, double dt,
                               const ot_force_schedule* pulls, const ot_record* rec, const float* dL_dtips,
                               ot_grads* grads, void* workspace, size_t workspace_bytes, void* stream) {
  StepArgs a{};
  BackArgs ba{};
  int ce = 0;
  ot_status st = backward_args(m, s, n_steps, step0, dt, pulls, rec, dL_dtips, grads, workspace, workspace_bytes,
                               &a, &ba, &ce);
  if (st != OT_OK) return st;
  cudaStream_t cs = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  OT_CUDA(cudaEventCreate(&e0));
  OT_CUDA(cudaEventCreate(&e1));
  ot_status result = OT_OK;
  for (int k = 0; k < (int)m->P.classes.size() && result == OT_OK; ++k) {
    ClassInfo& ci = m->P.classes[k];
    float* work = back_work(m, (float*)workspace, k, ce);
    const int keep = ci.back_tpw;
    float best = 1e30f;
    int best_t = keep;
    for (int t : kBackTpw) {
      ci.back_tpw = t;
      if (launch_back_class(m, s, k, a, ba, work, ce, cs) != cudaSuccess) continue;  // warm-up
      cudaEventRecord(e0, cs);
      const cudaError_t e = launch_back_class(m, s, k, a, ba, work, ce, cs);
      cudaEventRecord(e1, cs);
      if (e != cudaSuccess) continue;
      if (cudaEventSynchronize(e1) != cudaSuccess) {
        result = cuda_fail(cudaGetLastError());
        break;
      }
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) {
        best = ms;
        best_t = t;
      }
    }
    ci.back_tpw = best_t;
  }
  cudaGetLastError();  // a candidate that could not launch leaves no error behind
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return result;
}

ot_status ot_rollout_backward(ot_model* m, ot_state* s, int32_t n_steps, int32_t step0, double dt,
                              const ot_force_schedule* pulls, const ot_record* rec, const float* dL_dtips,
                              ot_grads* grads, void* workspace, size_t workspace_bytes, void* stream) {
  StepArgs a{};
  BackArgs ba{};
  int ce = 0;
  {
    const ot_status st = backward_args(m, s, n_steps, step0, dt, pulls, rec, dL_dtips, grads, workspace,
                                       workspace_bytes, &a, &ba, &ce);
    if (st != OT_OK) return st;
  }
  cudaStream_t cs = (cudaStream_t)stream;
  float* work = (float*)workspace;
  // the classes run concurrently: each on its own stream, forked from and joined back to `stream`
  const int nk = (int)m->P.classes.size();
  {
    const ot_status r = ensure_class_streams(m);
    if (r != OT_OK) return r;
  }
  OT_CUDA(cudaEventRecord(m->fork_event, cs));
  ot_status result = OT_OK;
  for (int k = nk - 1; k >= 0; --k) {
    cudaStream_t sk = m->class_streams[k];
    OT_CUDA(cudaStreamWaitEvent(sk, m->fork_event, 0));
    const cudaError_t e = launch_back_class(m, s, k, a, ba, back_work(m, work, k, ce), ce, sk);
    if (e != cudaSuccess && result == OT_OK) result = cuda_fail(e);
    // always join, so `stream` waits for whatever was enqueued
    OT_CUDA(cudaEventRecord(m->join_events[k], sk));
    OT_CUDA(cudaStreamWaitEvent(cs, m->join_events[k], 0));
  }
  if (result != OT_OK) return result;
  return OT_OK;
}

}  // extern "C"

// ------------------------------------------------------------------------------------------
// Helpers of ot_step_static_scratch (static_scratch.cu): the per-class launch of one step with
// the workspace in memory the caller of these helpers provides.
// ------------------------------------------------------------------------------------------
namespace orchard {

ot_status static_step_plan(ot_model* m, const ot_state* s, const ot_force_schedule* pulls, size_t scratch_floats,
                           int max_classes, int* n_classes, StaticShape* shapes) {
  if (!m || !s || s->model != m || !n_classes || !shapes) return OT_EINVAL;
  StepArgs probe{};
  if (fill_pulls(probe, pulls) != OT_OK) return OT_EINVAL;
  const int nk = (int)m->P.classes.size();
  if (nk > max_classes) return OT_ECAPACITY;
  for (int k = 0; k < nk; ++k) {
    const ClassInfo& ci = m->P.classes[k];
    if ((size_t)ci.ws_floats > scratch_floats) return OT_ECAPACITY;  // one world does not fit
  }
  for (int k = 0; k < nk; ++k) {
    const ClassInfo& ci = m->P.classes[k];
    const ot_schedule& sc = ci.sched;
    // every group needs a slot of its own: a block never holds more groups than the array
    // has slots (the class's own schedule may ask for more worlds per block)
    const long long slots = (long long)(scratch_floats / (size_t)ci.ws_floats);
    const int wpb = (int)std::min<long long>(sc.worlds_per_block, slots);
    int bps = 0;
    OT_CUDA(kernel_attributes(sc.threads_per_world, false, false, wpb, 1, &bps));
    if (bps < 1) return OT_ECAPACITY;
    const int worlds = ci.q_end - ci.q_begin;
    long long blocks = std::min<long long>((long long)bps * m->n_sm, (worlds + wpb - 1) / wpb);
    blocks = std::min<long long>(blocks, slots / wpb);
    if (blocks < 1 && worlds > 0) return OT_ECAPACITY;
    shapes[k].worlds_per_block = wpb;
    shapes[k].blocks = (int)blocks;
  }
  *n_classes = nk;
  return OT_OK;
}

ot_status static_step_class(ot_model* m, ot_state* s, int k, const StaticShape& sh, const float* ext_force,
                            const ot_force_schedule* pulls, int32_t step, double dt, float* scratch, int* counter,
                            void* stream) {
  const ClassInfo& ci = m->P.classes[k];
  if (sh.blocks < 1) return OT_OK;
  StepArgs a = base_args(m, dt);
  a.step0 = step;
  a.n_steps = 1;
  a.ext_force = ext_force;
  fill_pulls(a, pulls);  // validated by the plan
  a.q_begin = ci.q_begin;
  a.q_end = ci.q_end;
  a.q_counter = counter;
  a.ws_floats = ci.ws_floats;
  a.global_ws = 1;
  DevState ds = s->dev;
  ds.scratch = scratch;
  launch_rollout(ci.sched.threads_per_world, sh.worlds_per_block, sh.blocks, 0, (cudaStream_t)stream, m->dev, ds,
                 a);
  OT_CUDA(cudaGetLastError());
  g_launches += 1;
  return OT_OK;
}

}  // namespace orchard
