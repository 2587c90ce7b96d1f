// Host-side substructuring (Sec. 2, Sec. 3, Sec. 7.1).  See topology.h.
//
// Every lookup from a level dof to a position runs through dense scratch
// arrays over the level's dof space and every grouping through a sort, so
// the cost is linear (up to sorts) in the mesh and interface sizes.
#include "topology.h"

#include <algorithm>
#include <cstdlib>
#include <exception>
#include <map>
#include <stdexcept>
#include <string>
#include <thread>
#include <unordered_map>

#include "amb.h"
#include "common.h"

namespace amb {

namespace {

// f(t, i0, i1) on [0, n) cut into contiguous chunks, one per host thread (up
// to 16 and to AMB_HOST_THREADS, at least min_per_thread indices each, and no more than
// scratch_budget / scratch_bytes threads when each needs scratch_bytes of its
// own); t numbers the chunks.  Every index writes only its own outputs, so
// the result does not depend on the split.  An exception in a chunk is
// rethrown after all chunks end; chunks whose thread cannot be started run
// on the calling thread.
// AMB_HOST_THREADS (environment, read once) caps the thread count; 1 runs
// everything on the calling thread.
int host_thread_cap() {
  static const int cap = [] {
    const char* v = std::getenv("AMB_HOST_THREADS");
    const int n = v ? std::atoi(v) : 0;
    return n > 0 ? n : 16;
  }();
  return cap;
}

template <class F>
void parallel_chunks(int64_t n, int64_t min_per_thread, size_t scratch_bytes, F f) {
  const unsigned hw = std::thread::hardware_concurrency();
  int64_t nt = std::min<int64_t>(hw ? (int64_t)hw : 1, std::min(16, host_thread_cap()));
  nt = std::min<int64_t>(nt, std::max<int64_t>(1, n / std::max<int64_t>(min_per_thread, 1)));
  constexpr size_t kScratchBudget = size_t(256) << 20;
  if (scratch_bytes > 0) nt = std::min<int64_t>(nt, std::max<int64_t>(1, (int64_t)(kScratchBudget / scratch_bytes)));
  if (nt <= 1) {
    f(0, (int64_t)0, n);
    return;
  }
  std::vector<std::thread> th;
  th.reserve((size_t)nt);
  std::vector<std::exception_ptr> err((size_t)nt);
  auto chunk = [&f, &err, n, nt](int64_t t) {
    try {
      f((int)t, n * t / nt, n * (t + 1) / nt);
    } catch (...) {
      err[(size_t)t] = std::current_exception();
    }
  };
  int64_t started = 0;
  try {
    for (; started < nt; ++started) th.emplace_back(chunk, started);
  } catch (...) {
    // no thread could be started: the calling thread runs the remaining chunks
  }
  for (int64_t t = started; t < nt; ++t) chunk(t);
  for (auto& x : th) x.join();
  for (auto& e : err)
    if (e) std::rethrow_exception(e);
}

enum { TAG_X0 = 1, TAG_X1 = 2, TAG_Y0 = 4, TAG_Y1 = 8, TAG_Z0 = 16, TAG_Z1 = 32 };

// Nodes of a level (level 1: mesh nodes; level >= 2: coarse objects of the
// level below), in CSR form.
struct LevelNodes {
  int64_t n_dofs = 0;                         // level dof id space
  std::vector<int> soff{0}, subs;             // sharing substructures of each node, sorted
  std::vector<int> tags;                      // boundary bits of each node
  std::vector<char> eligible;                 // may be a corner
  std::vector<int64_t> doff{0}, dofs;         // level dofs of each node (none: no free dof)
  std::vector<int> comps;                     // component of each of those dofs (-1 scalar)
  int size() const { return (int)tags.size(); }
  int nsub(int i) const { return soff[i + 1] - soff[i]; }
  const int* sub(int i) const { return subs.data() + soff[i]; }
  int64_t ndof(int i) const { return doff[i + 1] - doff[i]; }
};

bool set_less(const LevelNodes& N, int a, int b) {
  return std::lexicographical_compare(N.sub(a), N.sub(a) + N.nsub(a), N.sub(b), N.sub(b) + N.nsub(b));
}
bool set_equal(const LevelNodes& N, int a, int b) {
  return N.nsub(a) == N.nsub(b) && std::equal(N.sub(a), N.sub(a) + N.nsub(a), N.sub(b));
}

// One arithmetic average per component over the dofs of `nodes` (an edge
// or a face: nodes with the same sharing set), weights 1/n (Sec. 7.1).
CoarseObj average_object(const LevelNodes& N, int kind, const std::vector<int>& nodes) {
  CoarseObj ob;
  ob.kind = kind;
  ob.subs.assign(N.sub(nodes[0]), N.sub(nodes[0]) + N.nsub(nodes[0]));
  int tags = ~0;
  std::map<int, std::vector<int64_t>> bycomp;
  for (int i : nodes) {
    tags &= N.tags[i];
    for (int64_t q = N.doff[i]; q < N.doff[i + 1]; ++q) {
      AMB_CHECK(N.comps[q] >= 0, AMB_EINVAL,
                kind == OBJ_EDGE ? "a scalar coarse dof lies on an edge of the next level"
                                 : "a scalar coarse dof lies on a face of the next level");
      bycomp[N.comps[q]].push_back(N.dofs[q]);
    }
  }
  ob.tags = tags;
  for (auto& c : bycomp) {
    std::sort(c.second.begin(), c.second.end());
    ob.comps.push_back(c.first);
    ob.w.push_back(std::vector<double>(c.second.size(), 1.0 / (double)c.second.size()));
    ob.dofs.push_back(c.second);
  }
  return ob;
}

// Classify the nodes of a level and build its substructures, objects and
// interface numbering.
void classify(LevelTopo& L, const LevelNodes& N, int initial) {
  const int nn = N.size();
  std::vector<char> iface(nn, 0), corner(nn, 0);
  std::vector<int> order;
  for (int i = 0; i < nn; ++i) {
    iface[i] = N.nsub(i) >= 2 && N.ndof(i) > 0;
    if (iface[i]) order.push_back(i);
  }
  // rank of each interface node's sharing set in lexicographic set order:
  // distinct sets by hashing, then only the distinct sets are sorted
  std::vector<int> rank(nn, -1);
  {
    std::unordered_map<uint64_t, std::vector<int>> buckets;   // hash -> distinct set ids
    std::vector<int> rep, sid(nn, -1);                         // representative node of each set
    for (int i : order) {
      uint64_t h = 1469598103934665603ull;
      for (int k = 0; k < N.nsub(i); ++k) h = (h ^ (uint64_t)(uint32_t)N.sub(i)[k]) * 1099511628211ull;
      auto& b = buckets[h];
      int id = -1;
      for (int r : b)
        if (set_equal(N, rep[r], i)) { id = r; break; }
      if (id < 0) {
        id = (int)rep.size();
        rep.push_back(i);
        b.push_back(id);
      }
      sid[i] = id;
    }
    std::vector<int> ord(rep.size()), rk(rep.size());
    for (size_t r = 0; r < rep.size(); ++r) ord[r] = (int)r;
    std::sort(ord.begin(), ord.end(), [&](int a, int b) { return set_less(N, rep[a], rep[b]); });
    for (size_t r = 0; r < ord.size(); ++r) rk[ord[r]] = (int)r;
    for (int i : order) rank[i] = rk[sid[i]];
  }
  // corner rule: a vertex of the box grid (with b boundary bits, shared by
  // 2^(3-b) substructures) that is alone in its (sharing set, tags) class
  auto box_vertex = [&](int i) {
    const int nb = __builtin_popcount((unsigned)N.tags[i] & 63u);
    return nb <= 3 && N.nsub(i) == (1 << (3 - nb));
  };
  // order by (rank, tags, node index): a stable counting sort of the nodes
  // (already in index order) on the key rank * ntag + tags
  int nrank = 0, ntag = 1;
  for (int i : order) {
    nrank = std::max(nrank, rank[i] + 1);
    AMB_CHECK(N.tags[i] >= 0, AMB_EINVAL, "negative node tags");
    ntag = std::max(ntag, N.tags[i] + 1);
  }
  auto counting_sort = [](std::vector<int>& v, int nkeys, auto key) {
    std::vector<int> start((size_t)nkeys + 1, 0), out(v.size());
    for (int i : v) ++start[key(i) + 1];
    for (int k = 0; k < nkeys; ++k) start[k + 1] += start[k];
    for (int i : v) out[start[key(i)]++] = i;
    v.swap(out);
  };
  counting_sort(order, nrank * ntag, [&](int i) { return rank[i] * ntag + N.tags[i]; });
  for (size_t r = 0; r < order.size();) {
    size_t e = r + 1;
    while (e < order.size() && rank[order[r]] == rank[order[e]] && N.tags[order[r]] == N.tags[order[e]]) ++e;
    if (e == r + 1 && N.eligible[order[r]] && box_vertex(order[r])) corner[order[r]] = 1;
    r = e;
  }
  // remaining interface nodes grouped by sharing set: sets in lexicographic
  // order, nodes in index order within a set
  std::vector<int> grp;
  for (int i = 0; i < nn; ++i)
    if (iface[i] && !corner[i]) grp.push_back(i);
  counting_sort(grp, nrank, [&](int i) { return rank[i]; });

  L.n_dofs = N.n_dofs;
  L.objs.clear();
  // corner objects, in node order
  for (int i = 0; i < nn; ++i) {
    if (!corner[i]) continue;
    CoarseObj ob;
    ob.kind = OBJ_CORNER;
    ob.subs.assign(N.sub(i), N.sub(i) + N.nsub(i));
    ob.tags = N.tags[i];
    ob.corner_node = i;
    for (int64_t q = N.doff[i]; q < N.doff[i + 1]; ++q) {
      ob.comps.push_back(N.comps[q]);
      ob.dofs.push_back({N.dofs[q]});
      ob.w.push_back({1.0});
    }
    L.objs.push_back(std::move(ob));
  }
  L.n_corner_nodes = (int)L.objs.size();
  // edges (sets of >= 3 substructures) in set order; faces (2 substructures)
  L.n_edges = 0;
  std::vector<std::pair<int, std::vector<int>>> faces;   // (first node of the set, nodes)
  for (size_t r = 0; r < grp.size();) {
    size_t e = r + 1;
    while (e < grp.size() && rank[grp[r]] == rank[grp[e]]) ++e;
    const int i0 = grp[r];
    if (N.nsub(i0) == 2) {
      faces.emplace_back(i0, std::vector<int>(grp.begin() + r, grp.begin() + e));
    } else {
      ++L.n_edges;
      if (initial == AMB_CORNERS_EDGES || initial == AMB_CORNERS_EDGES_FACES)
        L.objs.push_back(average_object(N, OBJ_EDGE, std::vector<int>(grp.begin() + r, grp.begin() + e)));
    }
    r = e;
  }
  L.n_faces = (int)faces.size();
  // face averages (Sec. 8.2, "c+e+f"), after the edges, in sharing-set order
  if (initial == AMB_CORNERS_EDGES_FACES)
    for (auto& f : faces) L.objs.push_back(average_object(N, OBJ_FACE, f.second));

  // substructure dof lists: interior, delta, corner (each sorted by level
  // dof), gathered in node order over node ranges in parallel: counts per
  // (range, kind, substructure), then every range fills its own slots
  L.subs.assign(L.n_subs, SubTopo());
  const int ns = L.n_subs;
  std::vector<std::vector<int64_t>> lists[3];   // interior, delta, corner
  for (auto& l : lists) l.assign(ns, {});
  auto kind_of = [&](int i) { return !iface[i] ? 0 : (corner[i] ? 2 : 1); };
  std::vector<std::vector<int64_t>> kcnt(16, std::vector<int64_t>());
  int nchunks = 0;
  parallel_chunks(nn, 1 << 14, 0, [&](int t, int64_t i0, int64_t i1) {
    std::vector<int64_t>& c = kcnt[t];
    c.assign((size_t)3 * ns, 0);
    for (int64_t i = i0; i < i1; ++i) {
      if (N.ndof((int)i) == 0) continue;
      const int kd = kind_of((int)i);
      for (int k = 0; k < N.nsub((int)i); ++k) c[(size_t)kd * ns + N.sub((int)i)[k]] += N.ndof((int)i);
    }
  });
  for (int t = 0; t < 16; ++t)
    if (!kcnt[t].empty()) nchunks = t + 1;
  std::vector<int64_t> base((size_t)nchunks * 3 * ns, 0);   // start of chunk t in each list
  for (int kd = 0; kd < 3; ++kd)
    for (int sb = 0; sb < ns; ++sb) {
      int64_t run = 0;
      for (int t = 0; t < nchunks; ++t) {
        base[((size_t)t * 3 + kd) * ns + sb] = run;
        run += kcnt[t][(size_t)kd * ns + sb];
      }
      lists[kd][sb].resize(run);
    }
  parallel_chunks(nn, 1 << 14, 0, [&](int t, int64_t i0, int64_t i1) {
    int64_t* pos = base.data() + (size_t)t * 3 * ns;
    for (int64_t i = i0; i < i1; ++i) {
      if (N.ndof((int)i) == 0) continue;
      const int kd = kind_of((int)i);
      for (int k = 0; k < N.nsub((int)i); ++k) {
        const int sb = N.sub((int)i)[k];
        int64_t& at = pos[(size_t)kd * ns + sb];
        std::copy(N.dofs.begin() + N.doff[i], N.dofs.begin() + N.doff[i + 1], lists[kd][sb].begin() + at);
        at += N.ndof((int)i);
      }
    }
  });
  std::vector<std::vector<int64_t>>& inter = lists[0];
  std::vector<std::vector<int64_t>>& delta = lists[1];
  std::vector<std::vector<int64_t>>& crn = lists[2];
  L.corner_dofs.clear();
  for (int i = 0; i < nn; ++i)
    if (corner[i]) L.corner_dofs.insert(L.corner_dofs.end(), N.dofs.begin() + N.doff[i], N.dofs.begin() + N.doff[i + 1]);
  std::sort(L.corner_dofs.begin(), L.corner_dofs.end());
  parallel_chunks(L.n_subs, 4, 0, [&](int, int64_t s0, int64_t s1) {
    for (int64_t s = s0; s < s1; ++s) {
      // in node order the lists are sorted already when a node's dofs are
      // consecutive and increasing with the node (level 1, and the coarse
      // dofs of the objects of a level below)
      for (auto* v : {&inter[s], &delta[s], &crn[s]})
        if (!std::is_sorted(v->begin(), v->end())) std::sort(v->begin(), v->end());
      SubTopo& sb = L.subs[s];
      sb.n_i = (int)inter[s].size();
      sb.n_g = (int)(delta[s].size() + crn[s].size());
      sb.n_crn = (int)crn[s].size();
      sb.dofs.reserve(inter[s].size() + sb.n_g);
      sb.dofs = inter[s];
      sb.dofs.insert(sb.dofs.end(), delta[s].begin(), delta[s].end());
      sb.dofs.insert(sb.dofs.end(), crn[s].begin(), crn[s].end());
    }
  });
  // global interface numbering (increasing level dof) and owners (increasing
  // substructure), by counting over the level's dof space
  std::vector<int> cnt(N.n_dofs + 1, 0);
  for (int s = 0; s < L.n_subs; ++s) {
    const SubTopo& sb = L.subs[s];
    for (int l = 0; l < sb.n_g; ++l) ++cnt[sb.dofs[sb.n_i + l]];
  }
  L.iface_dofs.clear();
  L.own_off.assign(1, 0);
  std::vector<int> slot(N.n_dofs, -1);   // level dof -> global interface index
  for (int64_t d = 0; d < N.n_dofs; ++d) {
    if (cnt[d] == 0) continue;
    slot[d] = (int)L.iface_dofs.size();
    L.iface_dofs.push_back(d);
    L.own_off.push_back(L.own_off.back() + cnt[d]);
  }
  L.own_sub.assign(L.own_off.back(), 0);
  L.own_pos.assign(L.own_off.back(), 0);
  std::vector<int> fill(L.iface_dofs.size(), 0);
  L.gidx.assign(L.n_subs, {});
  for (int s = 0; s < L.n_subs; ++s) {
    const SubTopo& sb = L.subs[s];
    L.gidx[s].assign(sb.n_g, -1);
    for (int l = 0; l < sb.n_g; ++l) {
      const int j = slot[sb.dofs[sb.n_i + l]];
      const int q = L.own_off[j] + fill[j]++;
      L.own_sub[q] = s;
      L.own_pos[q] = l;
      L.gidx[s][l] = j;
    }
  }
  // pairs: faces with at least one face-class dof, sorted by (s, t)
  L.pairs.clear();
  for (auto& f : faces) {
    PairTopo p;
    p.s = N.sub(f.first)[0];
    p.t = N.sub(f.first)[1];
    std::vector<int64_t> fd;
    for (int i : f.second) fd.insert(fd.end(), N.dofs.begin() + N.doff[i], N.dofs.begin() + N.doff[i + 1]);
    if (fd.empty()) continue;
    std::sort(fd.begin(), fd.end());
    p.face_dofs = fd;
    L.pairs.push_back(std::move(p));
  }
  std::sort(L.pairs.begin(), L.pairs.end(), [](const PairTopo& a, const PairTopo& b) {
    return a.s != b.s ? a.s < b.s : a.t < b.t;
  });
}

}  // namespace

// ------------------------------------------------------------------ numbering

void number_coarse(LevelTopo& L) {
  int64_t n = 0;
  for (auto& ob : L.objs) {
    ob.first = n;
    n += (int64_t)ob.dofs.size();
  }
  L.n_coarse = n;
  // object lists per substructure (increasing object index)
  std::vector<std::vector<int>> objs_of(L.n_subs);
  for (int o = 0; o < (int)L.objs.size(); ++o)
    for (int s : L.objs[o].subs) objs_of[s].push_back(o);
  // scratch over the level's dof space, reset after each use
  std::vector<int> gpos(L.n_dofs, -1);
  for (int s = 0; s < L.n_subs; ++s) {
    SubTopo& sb = L.subs[s];
    for (int l = 0; l < sb.n_g; ++l) gpos[sb.dofs[sb.n_i + l]] = l;
    std::vector<int64_t> cc(sb.n_crn, -1);   // coarse id of each corner position
    sb.rc.clear();
    sb.crows.clear();
    std::vector<int64_t> others;
    for (int o : objs_of[s]) {
      const CoarseObj& ob = L.objs[o];
      for (size_t q = 0; q < ob.dofs.size(); ++q) {
        if (ob.kind == OBJ_CORNER) {
          const int pos = gpos[ob.dofs[q][0]];
          if (pos >= sb.n_d()) cc[pos - sb.n_d()] = ob.first + (int64_t)q;
        } else {
          std::vector<std::pair<int, double>> row;
          row.reserve(ob.dofs[q].size());
          for (size_t e = 0; e < ob.dofs[q].size(); ++e) {
            const int pos = gpos[ob.dofs[q][e]];
            AMB_CHECK(pos >= 0, AMB_EINVAL, "constraint dof outside the interface");
            AMB_CHECK(pos < sb.n_d(), AMB_EINVAL, "non-corner constraint touches a corner dof");
            row.push_back({pos, ob.w[q][e]});
          }
          others.push_back(ob.first + (int64_t)q);
          sb.crows.push_back(std::move(row));
        }
      }
    }
    for (int l = 0; l < sb.n_crn; ++l) {
      AMB_CHECK(cc[l] >= 0, AMB_EINVAL, "corner dof without a coarse dof");
      sb.rc.push_back(cc[l]);
    }
    sb.rc.insert(sb.rc.end(), others.begin(), others.end());
    for (int l = 0; l < sb.n_g; ++l) gpos[sb.dofs[sb.n_i + l]] = -1;
  }
  // pair data (pairs in parallel, scratch over the dof space per thread)
  parallel_chunks((int64_t)L.pairs.size(), 16, (size_t)2 * L.n_dofs * sizeof(int), [&](int, int64_t p0, int64_t p1) {
  std::vector<int> pb(L.n_dofs, -1), fent(L.n_dofs, -1);
  std::vector<std::pair<int64_t, int>> adofs;
  for (int64_t pi = p0; pi < p1; ++pi) {
    PairTopo& p = L.pairs[pi];
    const SubTopo& a = L.subs[p.s];
    const SubTopo& b = L.subs[p.t];
    for (int l = 0; l < b.n_g; ++l) pb[b.dofs[b.n_i + l]] = l;
    // shared positions in increasing level-dof order
    adofs.clear();
    for (int l = 0; l < a.n_g; ++l) adofs.push_back({a.dofs[a.n_i + l], l});
    std::sort(adofs.begin(), adofs.end());
    p.ps.clear();
    p.pt.clear();
    for (const auto& dl : adofs) {
      const int lb = pb[dl.first];
      if (lb < 0) continue;
      fent[dl.first] = (int)p.ps.size();
      p.ps.push_back(dl.second);
      p.pt.push_back(lb);
    }
    p.face.clear();
    for (int64_t d : p.face_dofs) {
      AMB_CHECK(fent[d] >= 0, AMB_EINVAL, "face dof not shared by the pair");
      p.face.push_back(fent[d]);
    }
    // jump groups: initial objects (corners, edges) shared by both, in object order
    p.goff.assign(1, 0);
    p.gent.clear();
    p.gw.clear();
    for (int o : objs_of[p.s]) {
      const CoarseObj& ob = L.objs[o];
      if (ob.kind == OBJ_ADAPTIVE) continue;
      if (!std::binary_search(ob.subs.begin(), ob.subs.end(), p.t)) continue;
      for (size_t q = 0; q < ob.dofs.size(); ++q) {
        for (size_t e = 0; e < ob.dofs[q].size(); ++e) {
          const int f = fent[ob.dofs[q][e]];
          AMB_CHECK(f >= 0, AMB_EINVAL, "jump constraint dof not shared by the pair");
          p.gent.push_back(f);
          p.gw.push_back(ob.w[q][e]);
        }
        p.goff.push_back((int)p.gent.size());
      }
    }
    for (int l = 0; l < b.n_g; ++l) pb[b.dofs[b.n_i + l]] = -1;
    for (const auto& dl : adofs) fent[dl.first] = -1;
    // pair coarse space (initial coarse dofs of both substructures)
    std::map<int64_t, int> pc;
    for (int64_t c : a.rc) pc.emplace(c, 0);
    for (int64_t c : b.rc) pc.emplace(c, 0);
    int k = 0;
    for (auto& kv : pc) kv.second = k++;
    p.n_cpair = k;
    p.cmap_s.clear();
    p.cmap_t.clear();
    for (int64_t c : a.rc) p.cmap_s.push_back(pc[c]);
    for (int64_t c : b.rc) p.cmap_t.push_back(pc[c]);
  }
  });
  check_topology(L);
}

void check_topology(const LevelTopo& L) {
  auto need = [](bool ok, const char* what) {
    if (!ok) throw Error(AMB_EINVAL, std::string("internal topology check failed: ") + what);
  };
  const int64_t ni = (int64_t)L.iface_dofs.size();
  need((int)L.subs.size() == L.n_subs, "substructure count");
  need((int64_t)L.own_off.size() == ni + 1 && L.own_off[0] == 0, "owner offsets");
  need(L.own_sub.size() == (size_t)L.own_off.back() && L.own_pos.size() == L.own_sub.size(), "owner lists");
  need(L.gidx.size() == L.subs.size(), "interface index lists");
  for (int s = 0; s < L.n_subs; ++s) {
    const SubTopo& sb = L.subs[s];
    need(sb.n_i >= 0 && sb.n_crn >= 0 && sb.n_crn <= sb.n_g, "substructure sizes");
    need(sb.dofs.size() == (size_t)(sb.n_i + sb.n_g), "substructure dof list");
    for (int64_t d : sb.dofs) need(d >= 0 && d < L.n_dofs, "substructure dof out of range");
    need(L.gidx[s].size() == (size_t)sb.n_g, "interface index list length");
    for (int l = 0; l < sb.n_g; ++l) {
      const int j = L.gidx[s][l];
      need(j >= 0 && j < ni && L.iface_dofs[j] == sb.dofs[sb.n_i + l], "interface index");
    }
    need(sb.rc.size() == (size_t)sb.n_crn + sb.crows.size(), "coarse dof list");
    for (int64_t c : sb.rc) need(c >= 0 && c < L.n_coarse, "coarse dof out of range");
    for (const auto& row : sb.crows)
      for (const auto& e : row) need(e.first >= 0 && e.first < sb.n_d(), "constraint position out of range");
  }
  for (int64_t j = 0; j < ni; ++j) {
    need(L.iface_dofs[j] >= 0 && L.iface_dofs[j] < L.n_dofs, "interface dof out of range");
    need(L.own_off[j + 1] > L.own_off[j], "interface dof without owner");
    for (int q = L.own_off[j]; q < L.own_off[j + 1]; ++q) {
      const int s = L.own_sub[q], l = L.own_pos[q];
      need(s >= 0 && s < L.n_subs && l >= 0 && l < L.subs[s].n_g && L.gidx[s][l] == j, "interface owner");
    }
  }
  for (const PairTopo& p : L.pairs) {
    need(p.s >= 0 && p.s < L.n_subs && p.t >= 0 && p.t < L.n_subs && p.s != p.t, "pair substructures");
    const SubTopo& a = L.subs[p.s];
    const SubTopo& b = L.subs[p.t];
    need(p.ps.size() == p.pt.size(), "pair shared lists");
    const int nf = (int)p.ps.size();
    for (int k = 0; k < nf; ++k) {
      need(p.ps[k] >= 0 && p.ps[k] < a.n_g && p.pt[k] >= 0 && p.pt[k] < b.n_g, "pair shared position");
      need(a.dofs[a.n_i + p.ps[k]] == b.dofs[b.n_i + p.pt[k]], "pair shared dof");
    }
    need(p.face.size() == p.face_dofs.size(), "pair face list");
    for (int f : p.face) need(f >= 0 && f < nf, "pair face entry");
    need(!p.goff.empty() && p.goff[0] == 0 && (size_t)p.goff.back() == p.gent.size() &&
             p.gw.size() == p.gent.size(), "pair jump groups");
    for (size_t g = 1; g < p.goff.size(); ++g) need(p.goff[g] >= p.goff[g - 1], "pair jump group offsets");
    for (int e : p.gent) need(e >= 0 && e < nf, "pair jump entry");
    need(p.cmap_s.size() == a.rc.size() && p.cmap_t.size() == b.rc.size(), "pair coarse maps");
    for (int c : p.cmap_s) need(c >= 0 && c < p.n_cpair, "pair coarse index");
    for (int c : p.cmap_t) need(c >= 0 && c < p.n_cpair, "pair coarse index");
  }
  for (int64_t d : L.corner_dofs) need(d >= 0 && d < L.n_dofs, "corner dof out of range");
}

void add_adaptive_rows(LevelTopo& L, int pi, const std::vector<std::vector<double>>& rows) {
  const PairTopo& p = L.pairs[pi];
  for (const auto& r : rows) {
    CoarseObj ob;
    ob.kind = OBJ_ADAPTIVE;
    ob.subs = {p.s, p.t};
    ob.comps = {-1};
    ob.dofs = {p.face_dofs};
    ob.w = {r};
    ob.tags = 0;
    L.objs.push_back(std::move(ob));
  }
}

// ------------------------------------------------------------------ checks

void validate_partition(int nx, int ny, int nz, const int32_t* elem_to_sub,
                        const std::vector<std::vector<int32_t>>& parents, const std::vector<int>& nsubs) {
  struct Box {
    int64_t lo[3] = {INT64_MAX, INT64_MAX, INT64_MAX}, hi[3] = {-1, -1, -1};
    int64_t count = 0;
    void add(const Box& b) {
      for (int a = 0; a < 3; ++a) {
        lo[a] = std::min(lo[a], b.lo[a]);
        hi[a] = std::max(hi[a], b.hi[a]);
      }
      count += b.count;
    }
    int64_t volume() const { return (hi[0] - lo[0] + 1) * (hi[1] - lo[1] + 1) * (hi[2] - lo[2] + 1); }
  };
  auto check_boxes = [](const std::vector<Box>& boxes, int level) {
    for (size_t s = 0; s < boxes.size(); ++s) {
      AMB_CHECK(boxes[s].count > 0, AMB_EINVAL,
                "level-" + std::to_string(level) + " substructure " + std::to_string(s) + " is empty");
      AMB_CHECK(boxes[s].count == boxes[s].volume(), AMB_EINVAL,
                "level-" + std::to_string(level) + " substructure " + std::to_string(s) +
                    " is not a box of elements");
    }
  };
  const int n1 = nsubs.empty() ? 0 : nsubs[0];
  AMB_CHECK(n1 >= 1, AMB_EINVAL, "n_sub1 must be >= 1");
  std::vector<Box> boxes(n1);
  int64_t e = 0;
  for (int64_t k = 0; k < nz; ++k)
    for (int64_t j = 0; j < ny; ++j)
      for (int64_t i = 0; i < nx; ++i, ++e) {
        const int32_t s = elem_to_sub[e];
        AMB_CHECK(s >= 0 && s < n1, AMB_EINVAL, "elem_to_sub out of range");
        Box& b = boxes[s];
        const int64_t x[3] = {i, j, k};
        for (int a = 0; a < 3; ++a) {
          b.lo[a] = std::min(b.lo[a], x[a]);
          b.hi[a] = std::max(b.hi[a], x[a]);
        }
        ++b.count;
      }
  check_boxes(boxes, 1);
  for (size_t l = 0; l < parents.size(); ++l) {
    const int nn = nsubs[l + 1];
    AMB_CHECK(nn >= 1, AMB_EINVAL, "every level needs at least one substructure");
    AMB_CHECK(parents[l].size() == boxes.size(), AMB_EINVAL, "sub_to_parent has the wrong length");
    std::vector<Box> up(nn);
    for (size_t s = 0; s < boxes.size(); ++s) {
      const int32_t q = parents[l][s];
      AMB_CHECK(q >= 0 && q < nn, AMB_EINVAL, "sub_to_parent out of range");
      up[q].add(boxes[s]);
    }
    check_boxes(up, (int)l + 2);
    boxes.swap(up);
  }
}

// ------------------------------------------------------------------ level 1

LevelTopo build_level_one(int nx, int ny, int nz, int dpn, const uint8_t* dirichlet, const int32_t* elem_to_sub,
                          int n_subs, int initial, std::vector<int32_t>& elem_local) {
  const int64_t nnx = nx + 1, nny = ny + 1, nnz = nz + 1;
  const int64_t nn = nnx * nny * nnz;
  const int64_t nel = (int64_t)nx * ny * nz;
  parallel_chunks(nel, 1 << 16, 0, [&](int, int64_t e0, int64_t e1) {
    for (int64_t e = e0; e < e1; ++e)
      AMB_CHECK(elem_to_sub[e] >= 0 && elem_to_sub[e] < n_subs, AMB_EINVAL, "elem_to_sub out of range");
  });
  // sharing set of node n: the substructures of the (up to 8) elements around it, sorted
  auto sharing = [&](int64_t n, int* set) {
    const int64_t i = n % nnx, j = (n / nnx) % nny, k = n / (nnx * nny);
    int c = 0;
    for (int64_t ek = k - 1; ek <= k; ++ek) {
      if (ek < 0 || ek >= nz) continue;
      for (int64_t ej = j - 1; ej <= j; ++ej) {
        if (ej < 0 || ej >= ny) continue;
        for (int64_t ei = i - 1; ei <= i; ++ei) {
          if (ei < 0 || ei >= nx) continue;
          const int sb = elem_to_sub[ei + nx * (ej + ny * ek)];
          if (std::find(set, set + c, sb) == set + c) set[c++] = sb;
        }
      }
    }
    for (int a = 1; a < c; ++a)   // insertion sort of at most 8 ids
      for (int b = a; b > 0 && set[b - 1] > set[b]; --b) std::swap(set[b - 1], set[b]);
    return c;
  };
  // CSR of the nodes in two passes over node ranges: sizes, then contents
  LevelNodes N;
  N.n_dofs = nn * dpn;
  N.tags.assign(nn, 0);
  N.eligible.assign(nn, 1);
  N.soff.assign(nn + 1, 0);
  N.doff.assign(nn + 1, 0);
  parallel_chunks(nn, 1 << 14, 0, [&](int, int64_t n0, int64_t n1) {
    int set[8];
    for (int64_t n = n0; n < n1; ++n) {
      N.soff[n + 1] = sharing(n, set);
      N.doff[n + 1] = dirichlet[n] ? 0 : dpn;
    }
  });
  for (int64_t n = 0; n < nn; ++n) {
    N.soff[n + 1] += N.soff[n];
    N.doff[n + 1] += N.doff[n];
  }
  N.subs.resize(N.soff[nn]);
  N.dofs.resize(N.doff[nn]);
  N.comps.resize(N.doff[nn]);
  parallel_chunks(nn, 1 << 14, 0, [&](int, int64_t n0, int64_t n1) {
    int set[8];
    for (int64_t n = n0; n < n1; ++n) {
      const int c = sharing(n, set);
      std::copy(set, set + c, N.subs.begin() + N.soff[n]);
      const int64_t i = n % nnx, j = (n / nnx) % nny, k = n / (nnx * nny);
      int t = 0;
      if (i == 0) t |= TAG_X0;
      if (i == nx) t |= TAG_X1;
      if (j == 0) t |= TAG_Y0;
      if (j == ny) t |= TAG_Y1;
      if (k == 0) t |= TAG_Z0;
      if (k == nz) t |= TAG_Z1;
      N.tags[n] = t;
      for (int64_t q = N.doff[n]; q < N.doff[n + 1]; ++q) {
        N.dofs[q] = n * dpn + (q - N.doff[n]);
        N.comps[q] = (int)(q - N.doff[n]);
      }
    }
  });
  LevelTopo L;
  L.n_subs = n_subs;
  classify(L, N, initial);
  L.node_tags_of_obj.clear();
  for (auto& ob : L.objs) L.node_tags_of_obj.push_back(ob.tags);
  number_coarse(L);
  // element -> local index in its substructure, -1 for Dirichlet dofs
  const int nd = 8 * dpn;
  elem_local.assign(nel * nd, -1);
  std::vector<int64_t> eoff(n_subs + 1, 0), elems(nel);
  for (int64_t e = 0; e < nel; ++e) ++eoff[elem_to_sub[e] + 1];
  for (int s = 0; s < n_subs; ++s) eoff[s + 1] += eoff[s];
  {
    std::vector<int64_t> cur(eoff.begin(), eoff.end() - 1);
    for (int64_t e = 0; e < nel; ++e) elems[cur[elem_to_sub[e]]++] = e;
  }
  // substructures in parallel, each thread with its own dof -> position scratch
  parallel_chunks(n_subs, 2, (size_t)nn * dpn * sizeof(int32_t), [&](int, int64_t s0, int64_t s1) {
    std::vector<int32_t> loc(nn * dpn, -1);
    for (int64_t s = s0; s < s1; ++s) {
      const SubTopo& sb = L.subs[s];
      for (size_t q = 0; q < sb.dofs.size(); ++q) loc[sb.dofs[q]] = (int32_t)q;
      for (int64_t x = eoff[s]; x < eoff[s + 1]; ++x) {
        const int64_t e = elems[x];
        const int64_t i = e % nx, j = (e / nx) % ny, k = e / ((int64_t)nx * ny);
        for (int a = 0; a < 8; ++a) {
          const int64_t n = (i + (a & 1)) + nnx * ((j + ((a >> 1) & 1)) + nny * (k + ((a >> 2) & 1)));
          if (dirichlet[n]) continue;
          for (int c = 0; c < dpn; ++c) elem_local[e * nd + a * dpn + c] = loc[n * dpn + c];
        }
      }
      for (size_t q = 0; q < sb.dofs.size(); ++q) loc[sb.dofs[q]] = -1;
    }
  });
  return L;
}

// ------------------------------------------------------------------ level i+1

LevelTopo build_level_next(const LevelTopo& prev, const int32_t* parent, int n_subs, int initial,
                           std::vector<int32_t>& elem_local) {
  LevelNodes N;
  N.n_dofs = prev.n_coarse;
  const int no = (int)prev.objs.size();
  N.tags.assign(no, 0);
  N.eligible.assign(no, 0);
  for (int o = 0; o < no; ++o) {
    const CoarseObj& ob = prev.objs[o];
    std::vector<int> ps;
    for (int s : ob.subs) {
      AMB_CHECK(parent[s] >= 0 && parent[s] < n_subs, AMB_EINVAL, "sub_to_parent out of range");
      ps.push_back(parent[s]);
    }
    std::sort(ps.begin(), ps.end());
    ps.erase(std::unique(ps.begin(), ps.end()), ps.end());
    N.subs.insert(N.subs.end(), ps.begin(), ps.end());
    N.soff.push_back((int)N.subs.size());
    N.tags[o] = ob.tags;
    N.eligible[o] = ob.kind == OBJ_CORNER;
    for (size_t q = 0; q < ob.dofs.size(); ++q) {
      N.dofs.push_back(ob.first + (int64_t)q);
      N.comps.push_back(ob.comps[q]);
    }
    N.doff.push_back((int64_t)N.dofs.size());
  }
  LevelTopo L;
  L.n_subs = n_subs;
  classify(L, N, initial);
  number_coarse(L);
  // element (level-i substructure) -> local index of each of its coarse dofs in the parent
  elem_local.clear();
  std::vector<int32_t> loc(prev.n_coarse, -1);
  std::vector<std::vector<int>> kids(n_subs);
  for (int s = 0; s < prev.n_subs; ++s) kids[parent[s]].push_back(s);
  std::vector<std::vector<int32_t>> per(prev.n_subs);
  for (int P = 0; P < n_subs; ++P) {
    const SubTopo& sb = L.subs[P];
    for (size_t q = 0; q < sb.dofs.size(); ++q) loc[sb.dofs[q]] = (int32_t)q;
    for (int s : kids[P]) {
      for (int64_t c : prev.subs[s].rc) {
        AMB_CHECK(loc[c] >= 0, AMB_EINVAL, "coarse dof outside its parent substructure");
        per[s].push_back(loc[c]);
      }
    }
    for (size_t q = 0; q < sb.dofs.size(); ++q) loc[sb.dofs[q]] = -1;
  }
  for (int s = 0; s < prev.n_subs; ++s) elem_local.insert(elem_local.end(), per[s].begin(), per[s].end());
  return L;
}

}  // namespace amb
