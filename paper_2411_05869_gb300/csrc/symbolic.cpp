// symbolic.cpp -- step A6: symbolic analysis of P C_z P^T and the frontal plan of the numeric factorization.
//
// The ordering P is the nested-dissection order of A5 relabelled by a postorder of its elimination tree
// (children in increasing index order, roots in increasing order): the fill is unchanged and every subtree
// becomes a contiguous column range, so chains of the tree turn into supernodes.
//
// The paper factors nothing at large N (Sec. 3.3 uses Lanczos and MINRES; the Discussion names a sparse
// Cholesky as the exact alternative); this is the build's own analysis, run once per point set:
//   * elimination tree by Liu's algorithm (union-find with path compression over the lower adjacency);
//   * exact column counts eta_j by the row-subtree skeleton method of Gilbert, Ng and Peyton (1994):
//     each row subtree T_i contributes +1 at its leaves and -1 at the least common ancestor of consecutive
//     leaves in postorder; eta_j is the subtree sum of these weights (minus one per child, plus one per leaf);
//   * fundamental supernodes (parent(j) = j+1, eta_j = eta_{j+1} + 1, j the only child of j+1), then relaxed
//     amalgamation in increasing column order: the supernode ending right before p merges into p when p is its
//     supernodal parent and either the merged width is <= 16 or the merged panel holds at most 10 % explicit
//     zeros (a bound on the total, so merges along a chain of separators cannot compound);
//   * row structure of every supernode, frontal row lists, extend-add relative indices, supernode levels,
//     an update-matrix memory plan (first fit, freed once the parent level has assembled), and the per-level
//     launch schedule of the numeric kernels.
#include <algorithm>
#include <cstring>
#include <map>
#include <stdexcept>

#include "gp_internal.cuh"

namespace {

struct FirstFit {
  std::map<int64_t, int64_t> free_;   // offset -> size
  int64_t top = 0, peak = 0;
  int64_t alloc(int64_t sz) {
    if (sz == 0) return 0;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= sz) {
        int64_t off = it->first, rem = it->second - sz;
        free_.erase(it);
        if (rem > 0) free_[off + sz] = rem;
        return off;
      }
    }
    int64_t off = top;
    top += sz;
    peak = std::max(peak, top);
    return off;
  }
  void release(int64_t off, int64_t sz) {
    if (sz == 0) return;
    auto it = free_.emplace(off, sz).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
        it = pv;
      }
    }
    if (it->first + it->second == top) {
      top = it->first;
      free_.erase(it);
    }
  }
};

inline int64_t tri(int64_t k) { return k * (k + 1) / 2; }

}  // namespace

void build_symbolic(int64_t n, const int64_t* rowptr, const int32_t* col, const int32_t* nd_perm, SymPlan& sp) {
  sp = SymPlan();
  sp.n = n;
  std::vector<int32_t>& perm = sp.perm;
  perm.assign(nd_perm, nd_perm + n);
  std::vector<int32_t> pinv(n);
  for (int64_t i = 0; i < n; i++) pinv[perm[i]] = (int32_t)i;

  // ---- elimination tree (Liu)
  std::vector<int32_t>& parent = sp.parent;
  parent.assign(n, -1);
  {
    std::vector<int32_t> anc(n, -1);
    for (int64_t i = 0; i < n; i++) {
      int32_t oi = perm[i];
      for (int64_t e = rowptr[oi]; e < rowptr[oi + 1]; e++) {
        int32_t r = pinv[col[e]];
        if (r >= i) continue;
        while (anc[r] != -1 && anc[r] != i) {
          int32_t t = anc[r];
          anc[r] = (int32_t)i;
          r = t;
        }
        if (anc[r] == -1) {
          anc[r] = (int32_t)i;
          parent[r] = (int32_t)i;
        }
      }
    }
  }

  // ---- postorder (children visited in increasing order)
  std::vector<int32_t> head(n, -1), next(n, -1), post(n), ipost(n);
  for (int64_t j = n - 1; j >= 0; j--)
    if (parent[j] >= 0) {
      next[j] = head[parent[j]];
      head[parent[j]] = (int32_t)j;
    }
  {
    std::vector<int32_t> stack;
    stack.reserve(64);
    int64_t k = 0;
    std::vector<int32_t> cursor(head);
    for (int64_t root = 0; root < n; root++) {
      if (parent[root] != -1) continue;
      stack.push_back((int32_t)root);
      while (!stack.empty()) {
        int32_t v = stack.back();
        int32_t c = cursor[v];
        if (c != -1) {
          cursor[v] = next[c];
          stack.push_back(c);
        } else {
          stack.pop_back();
          post[k] = v;
          ipost[v] = (int32_t)k;
          k++;
        }
      }
    }
  }

  // ---- relabel by the postorder: same fill, every subtree contiguous, chains become runs j, j+1, ...
  {
    std::vector<int32_t> p2(n), par2(n);
    for (int64_t k = 0; k < n; k++) p2[k] = perm[post[k]];
    for (int64_t j = 0; j < n; j++) par2[ipost[j]] = parent[j] >= 0 ? ipost[parent[j]] : -1;
    perm.swap(p2);
    parent.swap(par2);
    for (int64_t i = 0; i < n; i++) {
      pinv[perm[i]] = (int32_t)i;
      post[i] = (int32_t)i;
      ipost[i] = (int32_t)i;
    }
  }

  // ---- column counts (row-subtree skeleton weights)
  std::vector<int32_t>& eta = sp.eta;
  {
    std::vector<int32_t> first(n, -1), delta(n, 0), prevnbr(n, -1), prevleaf(n, -1), uf(n);
    for (int64_t k = 0; k < n; k++) {
      int32_t j = post[k];
      for (int32_t x = j; x != -1 && first[x] == -1; x = parent[x]) first[x] = (int32_t)k;
    }
    for (int64_t j = 0; j < n; j++) {
      uf[j] = (int32_t)j;
      if (first[j] == ipost[j]) delta[j] = 1;        // etree leaf: T_j = {j}
      if (parent[j] >= 0) delta[parent[j]] -= 1;
    }
    auto find = [&](int32_t x) {
      int32_t r = x;
      while (uf[r] != r) r = uf[r];
      while (uf[x] != r) {
        int32_t t = uf[x];
        uf[x] = r;
        x = t;
      }
      return r;
    };
    for (int64_t k = 0; k < n; k++) {
      int32_t j = post[k];
      int32_t oj = perm[j];
      for (int64_t e = rowptr[oj]; e < rowptr[oj + 1]; e++) {
        int32_t i = pinv[col[e]];
        if (i <= j) continue;
        if (prevnbr[i] < first[j]) {                   // j is a leaf of the row subtree T_i
          delta[j] += 1;
          if (prevleaf[i] != -1) delta[find(prevleaf[i])] -= 1;
          prevleaf[i] = j;
        }
        prevnbr[i] = (int32_t)k;
      }
      if (parent[j] >= 0) uf[j] = parent[j];
    }
    eta.assign(delta.begin(), delta.end());
    for (int64_t k = 0; k < n; k++) {
      int32_t j = post[k];
      if (parent[j] >= 0) eta[parent[j]] += eta[j];
    }
  }
  sp.nnzL = 0;
  sp.flops = 0.0;
  for (int64_t j = 0; j < n; j++) {
    sp.nnzL += eta[j];
    sp.flops += (double)eta[j] * (double)eta[j];
  }

  // ---- fundamental supernodes
  std::vector<int32_t> nchild(n, 0);
  for (int64_t j = 0; j < n; j++)
    if (parent[j] >= 0) nchild[parent[j]]++;
  std::vector<int64_t> fstart;
  fstart.push_back(0);
  for (int64_t j = 0; j + 1 < n; j++) {
    bool same = parent[j] == j + 1 && eta[j] == eta[j + 1] + 1 && nchild[j + 1] == 1;
    if (!same) fstart.push_back(j + 1);
  }
  fstart.push_back(n);

  // ---- relaxed amalgamation (stack of merged supernodes in column order)
  auto panel = [](int64_t f, int64_t l, int64_t r) { return tri(l - f + 1) + (l - f + 1) * r; };
  struct SN { int64_t f, l, exact, zeros; };
  std::vector<SN> stk;
  for (size_t s = 0; s + 1 < fstart.size(); s++) {
    SN p{fstart[s], fstart[s + 1] - 1, 0, 0};
    for (int64_t j = p.f; j <= p.l; j++) p.exact += eta[j];
    p.zeros = panel(p.f, p.l, eta[p.l] - 1) - p.exact;
    while (!stk.empty()) {
      const SN& c = stk.back();
      if (c.l != p.f - 1) break;
      int32_t par = parent[c.l];
      if (!(par >= p.f && par <= p.l)) break;
      int64_t ent = panel(c.f, p.l, eta[p.l] - 1);
      int64_t ex = c.exact + p.exact;
      int64_t mz = ent - ex;
      if (p.l - c.f + 1 <= GP_RELAX_WIDTH || 10 * mz <= ent) {
        p = SN{c.f, p.l, ex, mz};
        stk.pop_back();
      } else {
        break;
      }
    }
    stk.push_back(p);
  }
  const int64_t ns = (int64_t)stk.size();
  sp.ns = ns;
  sp.sn_first.resize(ns + 1);
  for (int64_t s = 0; s < ns; s++) sp.sn_first[s] = (int32_t)stk[s].f;
  sp.sn_first[ns] = (int32_t)n;
  sp.sn_of_col.resize(n);
  for (int64_t s = 0; s < ns; s++)
    for (int64_t j = sp.sn_first[s]; j < sp.sn_first[s + 1]; j++) sp.sn_of_col[j] = (int32_t)s;
  sp.sn_parent.resize(ns);
  sp.sn_w.resize(ns);
  for (int64_t s = 0; s < ns; s++) {
    int64_t l = sp.sn_first[s + 1] - 1;
    sp.sn_parent[s] = parent[l] >= 0 ? sp.sn_of_col[parent[l]] : -1;
    sp.sn_w[s] = sp.sn_first[s + 1] - sp.sn_first[s];
  }
  sp.ch_ptr.assign(ns + 1, 0);
  for (int64_t s = 0; s < ns; s++)
    if (sp.sn_parent[s] >= 0) sp.ch_ptr[sp.sn_parent[s] + 1]++;
  for (int64_t s = 0; s < ns; s++) sp.ch_ptr[s + 1] += sp.ch_ptr[s];
  sp.ch_idx.resize(sp.ch_ptr[ns]);
  {
    std::vector<int32_t> fill(sp.ch_ptr.begin(), sp.ch_ptr.end() - 1);
    for (int64_t s = 0; s < ns; s++)
      if (sp.sn_parent[s] >= 0) sp.ch_idx[fill[sp.sn_parent[s]]++] = (int32_t)s;
  }

  // ---- row structures (bottom-up unions)
  sp.sn_rowptr.assign(ns + 1, 0);
  sp.sn_rows.clear();
  {
    std::vector<int32_t> mark(n, -1), buf;
    for (int64_t s = 0; s < ns; s++) {
      int64_t f = sp.sn_first[s], l = sp.sn_first[s + 1] - 1;
      buf.clear();
      for (int64_t j = f; j <= l; j++) {
        int32_t oj = perm[j];
        for (int64_t e = rowptr[oj]; e < rowptr[oj + 1]; e++) {
          int32_t i = pinv[col[e]];
          if (i > l && mark[i] != s) {
            mark[i] = (int32_t)s;
            buf.push_back(i);
          }
        }
      }
      for (int32_t q = sp.ch_ptr[s]; q < sp.ch_ptr[s + 1]; q++) {
        int32_t c = sp.ch_idx[q];
        for (int64_t t = sp.sn_rowptr[c]; t < sp.sn_rowptr[c + 1]; t++) {
          int32_t i = sp.sn_rows[t];
          if (i > l && mark[i] != s) {
            mark[i] = (int32_t)s;
            buf.push_back(i);
          }
        }
      }
      std::sort(buf.begin(), buf.end());
      if ((int64_t)buf.size() != eta[l] - 1)
        throw GpError{GP_ERR_STATE, "symbolic analysis: supernode row count disagrees with column count"};
      sp.sn_rows.insert(sp.sn_rows.end(), buf.begin(), buf.end());
      sp.sn_rowptr[s + 1] = (int64_t)sp.sn_rows.size();
    }
  }

  // ---- frontal plan
  sp.sn_r.resize(ns);
  sp.sn_loff.resize(ns);
  sp.sn_frow.resize(ns + 1);
  sp.relidx_off.assign(ns + 1, 0);
  int64_t loff = 0, froff = 0;
  sp.max_front = 0;
  for (int64_t s = 0; s < ns; s++) {
    int64_t w = sp.sn_w[s], r = sp.sn_rowptr[s + 1] - sp.sn_rowptr[s];
    sp.sn_r[s] = (int32_t)r;
    sp.sn_loff[s] = loff;
    loff += (w + r) * w;
    sp.sn_frow[s] = froff;
    froff += w + r;
    sp.max_front = std::max<int32_t>(sp.max_front, (int32_t)(w + r));
  }
  sp.sn_frow[ns] = froff;
  sp.panel_entries = loff;
  sp.sn_ldw.resize(ns);
  sp.sn_loff32.resize(ns);
  sp.sn_doff.resize(ns);
  {
    int64_t o32 = 0, od = 0;
    for (int64_t s = 0; s < ns; s++) {
      int64_t w = sp.sn_w[s], m = w + sp.sn_r[s];
      int64_t ldw = (w + 3) / 4 * 4;
      sp.sn_ldw[s] = (int32_t)ldw;
      sp.sn_loff32[s] = o32;
      o32 += (m * ldw + 3) / 4 * 4;
      sp.sn_doff[s] = od;
      od += (w + GP_TILE - 1) / GP_TILE * GP_TILE * GP_TILE;
    }
    sp.panel32_entries = o32;
    sp.diag_entries = std::max<int64_t>(od, 1);
  }
  sp.frows.resize(froff);
  for (int64_t s = 0; s < ns; s++) {
    int64_t f = sp.sn_first[s], w = sp.sn_w[s];
    int32_t* fr = sp.frows.data() + sp.sn_frow[s];
    for (int64_t j = 0; j < w; j++) fr[j] = (int32_t)(f + j);
    std::copy(sp.sn_rows.begin() + sp.sn_rowptr[s], sp.sn_rows.begin() + sp.sn_rowptr[s + 1], fr + w);
  }
  sp.relidx.resize(sp.sn_rows.size());
  sp.vec_update_entries = (int64_t)sp.sn_rows.size();
  for (int64_t s = 0; s < ns; s++) {
    sp.relidx_off[s] = sp.sn_rowptr[s];
    int32_t p = sp.sn_parent[s];
    int64_t r = sp.sn_r[s];
    if (r == 0) continue;
    if (p < 0) throw GpError{GP_ERR_STATE, "symbolic analysis: root supernode with rows below"};
    const int32_t* pr = sp.frows.data() + sp.sn_frow[p];
    int64_t pm = sp.sn_w[p] + sp.sn_r[p];
    for (int64_t a = 0; a < r; a++) {
      int32_t row = sp.sn_rows[sp.sn_rowptr[s] + a];
      const int32_t* it = std::lower_bound(pr, pr + pm, row);
      if (it == pr + pm || *it != row)
        throw GpError{GP_ERR_STATE, "symbolic analysis: child row missing from parent front"};
      sp.relidx[sp.sn_rowptr[s] + a] = (int32_t)(it - pr);
    }
  }
  sp.relidx_off[ns] = (int64_t)sp.sn_rows.size();

  // ---- levels
  sp.sn_level.assign(ns, 0);
  for (int64_t s = 0; s < ns; s++)
    if (sp.sn_parent[s] >= 0)
      sp.sn_level[sp.sn_parent[s]] = std::max(sp.sn_level[sp.sn_parent[s]], sp.sn_level[s] + 1);
  sp.nlevels = 0;
  for (int64_t s = 0; s < ns; s++) sp.nlevels = std::max(sp.nlevels, sp.sn_level[s] + 1);
  sp.lev_ptr.assign(sp.nlevels + 1, 0);
  for (int64_t s = 0; s < ns; s++) sp.lev_ptr[sp.sn_level[s] + 1]++;
  for (int32_t l = 0; l < sp.nlevels; l++) sp.lev_ptr[l + 1] += sp.lev_ptr[l];
  sp.lev_sn.resize(ns);
  {
    std::vector<int32_t> fill(sp.lev_ptr.begin(), sp.lev_ptr.end() - 1);
    for (int64_t s = 0; s < ns; s++) sp.lev_sn[fill[sp.sn_level[s]]++] = (int32_t)s;
  }

  // ---- update-matrix memory plan: U_s allocated before its level's extend-add, freed after its parent's
  sp.sn_uoff.assign(ns, 0);
  {
    FirstFit ff;
    for (int32_t L = 0; L < sp.nlevels; L++) {
      for (int32_t q = sp.lev_ptr[L]; q < sp.lev_ptr[L + 1]; q++) {
        int32_t s = sp.lev_sn[q];
        int64_t r = sp.sn_r[s];
        sp.sn_uoff[s] = ff.alloc(r * r);
      }
      for (int32_t q = sp.lev_ptr[L]; q < sp.lev_ptr[L + 1]; q++) {
        int32_t s = sp.lev_sn[q];
        for (int32_t c = sp.ch_ptr[s]; c < sp.ch_ptr[s + 1]; c++) {
          int32_t ch = sp.ch_idx[c];
          ff.release(sp.sn_uoff[ch], (int64_t)sp.sn_r[ch] * sp.sn_r[ch]);
        }
      }
    }
    sp.update_entries = std::max<int64_t>(ff.peak, 1);
  }

  // ---- launch schedule
  sp.levels.assign(sp.nlevels, SymPlan::Level());
  sp.sn_lo_off.assign(sp.ns, 0);
  sp.lo_entries = 8;
  sp.level_large.assign(sp.nlevels, SymPlan::LevelLarge());
  sp.sn_fl.assign(sp.ns, -1);
  sp.n_fl = 0;
  sp.flow_fwd.clear();
  sp.flow_bwd.clear();
  sp.flow_fwd_ptr.assign(1, 0);
  sp.flow_bwd_ptr.assign(1, 0);
  for (int32_t L = 0; L < sp.nlevels; L++) {
    SymPlan::Level& lv = sp.levels[L];
    // extend-add: k-th child of every supernode of this level, 8 update columns per CTA
    int32_t maxch = 0;
    for (int32_t q = sp.lev_ptr[L]; q < sp.lev_ptr[L + 1]; q++) {
      int32_t s = sp.lev_sn[q];
      maxch = std::max(maxch, sp.ch_ptr[s + 1] - sp.ch_ptr[s]);
    }
    for (int32_t k = 0; k < maxch; k++) {
      SymPlan::EaLaunch ea{(int64_t)sp.ea_tab.size(), 0};
      for (int32_t q = sp.lev_ptr[L]; q < sp.lev_ptr[L + 1]; q++) {
        int32_t s = sp.lev_sn[q];
        if (sp.ch_ptr[s] + k >= sp.ch_ptr[s + 1]) continue;
        int32_t c = sp.ch_idx[sp.ch_ptr[s] + k];
        for (int32_t c0 = 0; c0 < sp.sn_r[c]; c0 += 8) sp.ea_tab.push_back(make_int2(c, c0));
      }
      ea.ncta = (int64_t)sp.ea_tab.size() - ea.tab_off;
      if (ea.ncta > 0) lv.ea.push_back(ea);
      SymPlan::EaLaunch e32{(int64_t)sp.ea32_tab.size(), 0};
      for (int32_t q = sp.lev_ptr[L]; q < sp.lev_ptr[L + 1]; q++) {
        int32_t s = sp.lev_sn[q];
        if (sp.ch_ptr[s] + k >= sp.ch_ptr[s + 1]) continue;
        int32_t c = sp.ch_idx[sp.ch_ptr[s] + k];
        const int64_t rc = sp.sn_r[c], nch = (rc * (rc + 1) / 2 + GP_EA_CHUNK - 1) / GP_EA_CHUNK;
        GP_REQUIRE(nch < INT32_MAX, "update matrix too large");
        for (int64_t h = 0; h < nch; h++) sp.ea32_tab.push_back(make_int2(c, (int)h));
      }
      e32.ncta = (int64_t)sp.ea32_tab.size() - e32.tab_off;
      if (e32.ncta > 0) lv.ea32.push_back(e32);
    }
    lv.zero_off = (int64_t)sp.zero_tab.size();
    for (int32_t q = sp.lev_ptr[L]; q < sp.lev_ptr[L + 1]; q++) {
      const int32_t s = sp.lev_sn[q];
      const int64_t r = sp.sn_r[s], nch = (r * (r + 1) / 2 + GP_EA_CHUNK - 1) / GP_EA_CHUNK;
      for (int64_t h = 0; h < nch; h++) sp.zero_tab.push_back(make_int2(s, (int)h));
    }
    lv.zero_n = (int64_t)sp.zero_tab.size() - lv.zero_off;
    // fronts
    lv.small_off = (int64_t)sp.small_list.size();
    std::vector<int32_t> large;
    for (int32_t q = sp.lev_ptr[L]; q < sp.lev_ptr[L + 1]; q++) {
      int32_t s = sp.lev_sn[q];
      if (sp.sn_w[s] + sp.sn_r[s] <= GP_SMALL_M) sp.small_list.push_back(s);
      else large.push_back(s);
    }
    lv.nsmall = (int32_t)((int64_t)sp.small_list.size() - lv.small_off);
    std::stable_sort(large.begin(), large.end(), [&](int32_t a, int32_t b) { return sp.sn_w[a] > sp.sn_w[b]; });
    sp.level_large[L].off = (int64_t)sp.large_fronts.size();
    if (!large.empty()) {
      int64_t maxw = sp.sn_w[large[0]];
      for (int32_t kb = 0; (int64_t)kb * GP_TILE < maxw; kb++) {
        SymPlan::StepLaunch stp{};
        stp.kb = kb;
        stp.fr_off = (int64_t)sp.large_fronts.size();
        stp.pre_off = (int64_t)sp.step_pre.size();
        int32_t cnt = 0;
        for (int32_t s : large)
          if ((int64_t)sp.sn_w[s] > (int64_t)kb * GP_TILE) {
            sp.large_fronts.push_back(s);
            sp.large_kb.push_back(kb);
            cnt++;
          }
        stp.nfront = cnt;
        // TRSM prefix then UPDATE prefix
        int64_t acc = 0;
        sp.step_pre.push_back(0);
        for (int32_t t = 0; t < cnt; t++) {
          int32_t s = sp.large_fronts[stp.fr_off + t];
          int64_t m = sp.sn_w[s] + sp.sn_r[s];
          int64_t c1 = std::min<int64_t>((int64_t)(kb + 1) * GP_TILE, sp.sn_w[s]);
          acc += (m - c1 + GP_TILE - 1) / GP_TILE;
          sp.step_pre.push_back(acc);
        }
        stp.trsm_total = acc;
        acc = 0;
        sp.step_pre.push_back(0);
        for (int32_t t = 0; t < cnt; t++) {
          int32_t s = sp.large_fronts[stp.fr_off + t];
          int64_t m = sp.sn_w[s] + sp.sn_r[s];
          int64_t c1 = std::min<int64_t>((int64_t)(kb + 1) * GP_TILE, sp.sn_w[s]);
          int64_t ntr = (m - c1 + GP_TILE - 1) / GP_TILE;
          acc += tri(ntr);
          sp.step_pre.push_back(acc);
        }
        stp.upd_total = acc;
        stp.potrf_flops = stp.trsm_flops = stp.upd_flops = 0.0;
        for (int32_t t = 0; t < cnt; t++) {
          int32_t s = sp.large_fronts[stp.fr_off + t];
          double m = (double)sp.sn_w[s] + sp.sn_r[s];
          double c0 = (double)kb * GP_TILE;
          double bw = std::min<double>(GP_TILE, sp.sn_w[s] - c0);
          double M = m - c0 - bw;
          stp.potrf_flops += bw * bw * bw / 3.0;
          stp.trsm_flops += M * bw * bw;
          stp.upd_flops += 2.0 * bw * M * (M + 1.0) / 2.0;
        }
        lv.steps.push_back(stp);
      }
      // The forward solve takes the steps two at a time (kb even, kb + 1): step kb + 1's fronts are the first
      // ones of step kb's (widths descending), and they apply both blocks to the rows after block kb + 1.
      for (size_t q = 0; q + 1 < lv.steps.size(); q += 2) {
        SymPlan::StepLaunch& s0 = lv.steps[q];
        const SymPlan::StepLaunch& s1 = lv.steps[q + 1];
        s0.pair_pre_off = (int64_t)sp.pair_pre.size();
        s0.pair_n2 = s1.nfront;
        int64_t acc = 0;
        sp.pair_pre.push_back(0);
        for (int32_t t = 0; t < s0.nfront; t++) {
          const int32_t s = sp.large_fronts[s0.fr_off + t];
          const int64_t w = sp.sn_w[s], m = w + sp.sn_r[s];
          const int64_t c1 = std::min<int64_t>((int64_t)(s0.kb + 1) * GP_TILE, w);
          const int64_t cs = t < s1.nfront ? std::min<int64_t>((int64_t)(s0.kb + 2) * GP_TILE, w) : c1;
          acc += (m - cs + GP_TILE - 1) / GP_TILE;
          sp.pair_pre.push_back(acc);
        }
        s0.pair_total = acc;
      }
    }
    sp.level_large[L].count = (int64_t)sp.large_fronts.size() - sp.level_large[L].off;
    // the tensor-core operands of this level's large fronts (the low TF32 parts, or the FP16 pairs): one region
    // per front in a workspace that every level reuses (read only by the updates of the front they belong to,
    // inside its level); m x ldh entries of 4 bytes, ldh = ldw rounded up to 8, so that the FP16 pair's rows
    // (ldh halves each) start on 16-byte boundaries
    {
      int64_t lo = 0;
      for (int32_t s : large) {
        sp.sn_lo_off[s] = lo;
        lo += (int64_t)(sp.sn_w[s] + sp.sn_r[s]) * ((sp.sn_ldw[s] + 7) / 8 * 8);
      }
      sp.lo_entries = std::max(sp.lo_entries, lo);
    }
    // dataflow solve tasks of this level's large fronts (SB blocks of 64 columns per chain task: 2 where the
    // level's chains are long, else 1; rows below the columns in tasks of 64 SB rows): forward tasks ordered by
    // their first block (the rows below a front's columns count as blocks nb, nb + 1, ...), backward tasks by
    // their distance from the last block; within either, the level's large-front order
    int64_t nbmax_l = 0;
    for (int32_t s : large) nbmax_l = std::max<int64_t>(nbmax_l, ((int64_t)sp.sn_w[s] + GP_TILE - 1) / GP_TILE);
    lv.flow_sb = nbmax_l >= GP_FLOW_SB_MIN_NB ? 2 : 1;
    const int64_t SBk = lv.flow_sb;
    int64_t imax = 0, nbsmax = 0;
    for (int32_t s : large) {
      const int64_t nb = ((int64_t)sp.sn_w[s] + GP_TILE - 1) / GP_TILE;
      sp.sn_fl[s] = (int32_t)sp.n_fl;
      sp.n_fl += nb;
      const int64_t nl = ((int64_t)sp.sn_r[s] + SBk * GP_TILE - 1) / (SBk * GP_TILE);
      imax = std::max<int64_t>(imax, nb + SBk * nl);
      nbsmax = std::max<int64_t>(nbsmax, (nb + SBk - 1) / SBk);
    }
    for (int64_t key = 0; key < imax; key++)
      for (int32_t s : large) {
        const int64_t nb = ((int64_t)sp.sn_w[s] + GP_TILE - 1) / GP_TILE, nbs = (nb + SBk - 1) / SBk;
        const int64_t nl = ((int64_t)sp.sn_r[s] + SBk * GP_TILE - 1) / (SBk * GP_TILE);
        if (key < nb) {
          if (key % SBk == 0) sp.flow_fwd.push_back(make_int2(s, (int)(key / SBk)));
        } else if ((key - nb) % SBk == 0 && (key - nb) / SBk < nl) {
          sp.flow_fwd.push_back(make_int2(s, (int)(nbs + (key - nb) / SBk)));
        }
      }
    for (int64_t d = 0; d < nbsmax; d++)
      for (int32_t s : large) {
        const int64_t nb = ((int64_t)sp.sn_w[s] + GP_TILE - 1) / GP_TILE, nbs = (nb + SBk - 1) / SBk;
        if (d < nbs) sp.flow_bwd.push_back(make_int2(s, (int)(nbs - 1 - d)));
      }
    sp.flow_fwd_ptr.push_back((int64_t)sp.flow_fwd.size());
    sp.flow_bwd_ptr.push_back((int64_t)sp.flow_bwd.size());
  }
  GP_REQUIRE(sp.n_fl < INT32_MAX, "too many solve blocks");
  plan_mixed_updates(sp, GP_GROUP, GP_TN_GROUP);
}

// The tensor-core update schedule of the mixed path for a given blocking: per step, the fronts (and tile
// prefixes) of the left-looking block-column update and, at a group's last block, of the group update.
//   group: 64-column blocks per group; tn: tile width (columns) of the group update, 128 or 256.
void plan_mixed_updates(SymPlan& sp, int group, int tn) {
  sp.group = group;
  sp.tn_group = tn;
  sp.upd_fronts.clear();
  sp.upd_pre.clear();
  for (auto& lv : sp.levels)
    for (auto& stp : lv.steps) {
      const int32_t kb = stp.kb, cnt = stp.nfront;
      stp.left_off = (int64_t)sp.upd_fronts.size();
      stp.left_pre_off = (int64_t)sp.upd_pre.size();
      stp.n_left = 0;
      stp.left_flops = 0.0;
      stp.left2_flops = 0.0;
      int64_t acc = 0;
      sp.upd_pre.push_back(0);
      std::vector<int64_t> rest_pre(1, 0);
      for (int32_t t = 0; t < cnt; t++) {   // block column kb from the earlier blocks of its group
        int32_t s = sp.large_fronts[stp.fr_off + t];
        int64_t w = sp.sn_w[s], m = w + sp.sn_r[s];
        int64_t c0 = (int64_t)kb * GP_TILE, c1 = std::min<int64_t>(c0 + GP_TILE, w);
        int64_t g0 = (int64_t)(kb / group) * group * GP_TILE;
        if (c0 == g0) continue;   // the first block of its group
        sp.upd_fronts.push_back(s);
        acc += (m - c0 + 127) / 128;
        sp.upd_pre.push_back(acc);
        rest_pre.push_back(rest_pre.back() + (m - c0 + 127) / 128 - 1);
        stp.n_left++;
        double bw = (double)(c1 - c0);
        stp.left_flops += 2.0 * (double)(c0 - g0) * (bw * (bw + 1.0) / 2.0 + (double)(m - c1) * bw);
        const int64_t c2 = std::min<int64_t>(c0 + 2 * GP_TILE, w);
        double cw = (double)(c2 - c0);
        stp.left2_flops += 2.0 * (double)(c0 - g0) * (cw * (cw + 1.0) / 2.0 + (double)(m - c2) * cw);
      }
      stp.left_total = acc;
      stp.lrest_pre_off = (int64_t)sp.upd_pre.size();
      stp.lrest_total = rest_pre.back();
      sp.upd_pre.insert(sp.upd_pre.end(), rest_pre.begin(), rest_pre.end());
      stp.group_off = (int64_t)sp.upd_fronts.size();
      stp.group_pre_off = (int64_t)sp.upd_pre.size();
      stp.n_group = 0;
      stp.group_flops = 0.0;
      acc = 0;
      sp.upd_pre.push_back(0);
      for (int32_t t = 0; t < cnt; t++) {   // fronts whose group ends at block kb: rows/columns after it
        int32_t s = sp.large_fronts[stp.fr_off + t];
        int64_t w = sp.sn_w[s], m = w + sp.sn_r[s];
        int64_t c1 = std::min<int64_t>((int64_t)(kb + 1) * GP_TILE, w);
        int64_t g0 = (int64_t)(kb / group) * group * GP_TILE;
        int64_t gend = std::min<int64_t>(g0 + (int64_t)group * GP_TILE, w);
        if (c1 < gend || gend >= m) continue;   // not a group end, or nothing after the group
        int64_t nt = (m - gend + 127) / 128;   // 128-row tile rows
        sp.upd_fronts.push_back(s);
        acc += tn == 256 ? tri((nt + 1) / 2) : tri(nt);   // 256 wide: tile pairs (rows 2p, 2p + 1)
        sp.upd_pre.push_back(acc);
        stp.n_group++;
        double M = (double)(m - gend);
        stp.group_flops += 2.0 * (double)(gend - g0) * M * (M + 1.0) / 2.0;
      }
      stp.group_total = acc;
    }
}
