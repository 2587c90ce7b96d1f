// Host-side substructuring (Sec. 2, Sec. 3, Sec. 7.1).  See topology.h.
#include "topology.h"

#include <algorithm>
#include <map>
#include <stdexcept>
#include <string>

#include "amb.h"
#include "common.h"

namespace amb {

namespace {

enum { TAG_X0 = 1, TAG_X1 = 2, TAG_Y0 = 4, TAG_Y1 = 8, TAG_Z0 = 16, TAG_Z1 = 32 };

// Classify the nodes of a level and build its substructures, objects and
// interface numbering.  node_elems_subs: per node its sharing set.
void classify(LevelTopo& L, const LevelNodes& N, int initial) {
  const int nn = (int)N.subs.size();
  std::vector<char> iface(nn, 0), corner(nn, 0);
  for (int i = 0; i < nn; ++i) iface[i] = N.subs[i].size() >= 2 && !N.dofs[i].empty();
  // corner rule: alone in its (sharing set, tags) class
  std::map<std::vector<int>, int> cls;
  auto key_of = [&](int i) {
    std::vector<int> k = N.subs[i];
    k.push_back(-1 - N.tags[i]);
    return k;
  };
  for (int i = 0; i < nn; ++i)
    if (iface[i]) cls[key_of(i)] += 1;
  for (int i = 0; i < nn; ++i)
    if (iface[i] && N.eligible[i] && cls[key_of(i)] == 1) corner[i] = 1;
  std::map<std::vector<int>, std::vector<int>> groups;
  for (int i = 0; i < nn; ++i)
    if (iface[i] && !corner[i]) groups[N.subs[i]].push_back(i);

  L.n_dofs = N.n_dofs;
  L.objs.clear();
  // corner objects, in node order
  std::vector<int> corner_obj(nn, -1);
  for (int i = 0; i < nn; ++i) {
    if (!corner[i]) continue;
    CoarseObj ob;
    ob.kind = OBJ_CORNER;
    ob.subs = N.subs[i];
    ob.tags = N.tags[i];
    ob.corner_node = i;
    for (size_t q = 0; q < N.dofs[i].size(); ++q) {
      ob.comps.push_back(N.comps[i][q]);
      ob.dofs.push_back({N.dofs[i][q]});
      ob.w.push_back({1.0});
    }
    corner_obj[i] = (int)L.objs.size();
    L.objs.push_back(std::move(ob));
  }
  L.n_corner_nodes = (int)L.objs.size();
  // edges (sets of >= 3 substructures), in key order
  L.n_edges = 0;
  L.n_faces = 0;
  std::vector<std::pair<std::vector<int>, std::vector<int>>> faces;
  for (auto& kv : groups) {
    if (kv.first.size() == 2) {
      faces.push_back(kv);
      continue;
    }
    ++L.n_edges;
    if (initial != AMB_CORNERS_EDGES) continue;
    CoarseObj ob;
    ob.kind = OBJ_EDGE;
    ob.subs = kv.first;
    int tags = ~0;
    std::map<int, std::vector<int64_t>> bycomp;
    for (int i : kv.second) {
      tags &= N.tags[i];
      for (size_t q = 0; q < N.dofs[i].size(); ++q) {
        AMB_CHECK(N.comps[i][q] >= 0, AMB_EINVAL, "a scalar coarse dof lies on an edge of the next level");
        bycomp[N.comps[i][q]].push_back(N.dofs[i][q]);
      }
    }
    ob.tags = tags;
    for (auto& c : bycomp) {
      std::sort(c.second.begin(), c.second.end());
      ob.comps.push_back(c.first);
      ob.w.push_back(std::vector<double>(c.second.size(), 1.0 / (double)c.second.size()));
      ob.dofs.push_back(c.second);
    }
    L.objs.push_back(std::move(ob));
  }
  L.n_faces = (int)faces.size();

  // substructure dof lists: interior, delta, corner (each sorted by level dof)
  L.subs.assign(L.n_subs, SubTopo());
  std::vector<std::vector<int64_t>> inter(L.n_subs), delta(L.n_subs), crn(L.n_subs);
  for (int i = 0; i < nn; ++i) {
    if (N.dofs[i].empty()) continue;
    for (int s : N.subs[i]) {
      auto& dst = !iface[i] ? inter[s] : (corner[i] ? crn[s] : delta[s]);
      for (int64_t d : N.dofs[i]) dst.push_back(d);
    }
  }
  L.corner_dofs.clear();
  for (int i = 0; i < nn; ++i)
    if (corner[i])
      for (int64_t d : N.dofs[i]) L.corner_dofs.push_back(d);
  std::sort(L.corner_dofs.begin(), L.corner_dofs.end());
  for (int s = 0; s < L.n_subs; ++s) {
    std::sort(inter[s].begin(), inter[s].end());
    std::sort(delta[s].begin(), delta[s].end());
    std::sort(crn[s].begin(), crn[s].end());
    SubTopo& sb = L.subs[s];
    sb.n_i = (int)inter[s].size();
    sb.n_g = (int)(delta[s].size() + crn[s].size());
    sb.n_crn = (int)crn[s].size();
    sb.dofs = inter[s];
    sb.dofs.insert(sb.dofs.end(), delta[s].begin(), delta[s].end());
    sb.dofs.insert(sb.dofs.end(), crn[s].begin(), crn[s].end());
  }
  // global interface numbering and owners
  std::map<int64_t, std::vector<std::pair<int, int>>> own;
  L.gidx.assign(L.n_subs, {});
  for (int s = 0; s < L.n_subs; ++s) {
    const SubTopo& sb = L.subs[s];
    for (int l = 0; l < sb.n_g; ++l) own[sb.dofs[sb.n_i + l]].push_back({s, l});
  }
  L.iface_dofs.clear();
  L.own_off.assign(1, 0);
  L.own_sub.clear();
  L.own_pos.clear();
  for (int s = 0; s < L.n_subs; ++s) L.gidx[s].assign(L.subs[s].n_g, -1);
  for (auto& kv : own) {
    int j = (int)L.iface_dofs.size();
    L.iface_dofs.push_back(kv.first);
    for (auto& sp : kv.second) {
      L.own_sub.push_back(sp.first);
      L.own_pos.push_back(sp.second);
      L.gidx[sp.first][sp.second] = j;
    }
    L.own_off.push_back((int)L.own_sub.size());
  }
  // pairs: faces with at least one face-class dof, sorted by (s, t)
  L.pairs.clear();
  for (auto& f : faces) {
    PairTopo p;
    p.s = f.first[0];
    p.t = f.first[1];
    std::vector<int64_t> fd;
    for (int i : f.second)
      for (int64_t d : N.dofs[i]) fd.push_back(d);
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
  // object lists per substructure
  std::vector<std::vector<int>> objs_of(L.n_subs);
  for (int o = 0; o < (int)L.objs.size(); ++o)
    for (int s : L.objs[o].subs) objs_of[s].push_back(o);
  for (int s = 0; s < L.n_subs; ++s) {
    SubTopo& sb = L.subs[s];
    std::map<int64_t, int> gpos;   // level dof -> interface position
    for (int l = 0; l < sb.n_g; ++l) gpos[sb.dofs[sb.n_i + l]] = l;
    std::map<int64_t, int64_t> corner_coarse;   // corner level dof -> coarse id
    sb.rc.clear();
    sb.crows.clear();
    std::vector<int64_t> others;
    for (int o : objs_of[s]) {
      const CoarseObj& ob = L.objs[o];
      for (size_t q = 0; q < ob.dofs.size(); ++q) {
        if (ob.kind == OBJ_CORNER) {
          corner_coarse[ob.dofs[q][0]] = ob.first + (int64_t)q;
        } else {
          std::vector<std::pair<int, double>> row;
          for (size_t e = 0; e < ob.dofs[q].size(); ++e) {
            auto it = gpos.find(ob.dofs[q][e]);
            AMB_CHECK(it != gpos.end(), AMB_EINVAL, "constraint dof outside the interface");
            int pos = it->second;   // interface position
            AMB_CHECK(pos < sb.n_d(), AMB_EINVAL, "non-corner constraint touches a corner dof");
            row.push_back({pos, ob.w[q][e]});
          }
          others.push_back(ob.first + (int64_t)q);
          sb.crows.push_back(std::move(row));
        }
      }
    }
    for (int l = sb.n_d(); l < sb.n_g; ++l) {
      auto it = corner_coarse.find(sb.dofs[sb.n_i + l]);
      AMB_CHECK(it != corner_coarse.end(), AMB_EINVAL, "corner dof without a coarse dof");
      sb.rc.push_back(it->second);
    }
    sb.rc.insert(sb.rc.end(), others.begin(), others.end());
  }
  // pair data
  for (auto& p : L.pairs) {
    const SubTopo& a = L.subs[p.s];
    const SubTopo& b = L.subs[p.t];
    std::map<int64_t, int> pa, pb;
    for (int l = 0; l < a.n_g; ++l) pa[a.dofs[a.n_i + l]] = l;
    for (int l = 0; l < b.n_g; ++l) pb[b.dofs[b.n_i + l]] = l;
    p.ps.clear();
    p.pt.clear();
    std::map<int64_t, int> fent;   // level dof -> entry index
    for (auto& kv : pa) {
      auto it = pb.find(kv.first);
      if (it == pb.end()) continue;
      fent[kv.first] = (int)p.ps.size();
      p.ps.push_back(kv.second);
      p.pt.push_back(it->second);
    }
    p.face.clear();
    for (int64_t d : p.face_dofs) {
      auto it = fent.find(d);
      AMB_CHECK(it != fent.end(), AMB_EINVAL, "face dof not shared by the pair");
      p.face.push_back(it->second);
    }
    // jump groups: initial objects (corners, edges) shared by both
    p.goff.assign(1, 0);
    p.gent.clear();
    p.gw.clear();
    for (const auto& ob : L.objs) {
      if (ob.kind == OBJ_ADAPTIVE) continue;
      if (!std::binary_search(ob.subs.begin(), ob.subs.end(), p.s) ||
          !std::binary_search(ob.subs.begin(), ob.subs.end(), p.t))
        continue;
      for (size_t q = 0; q < ob.dofs.size(); ++q) {
        for (size_t e = 0; e < ob.dofs[q].size(); ++e) {
          p.gent.push_back(fent.at(ob.dofs[q][e]));
          p.gw.push_back(ob.w[q][e]);
        }
        p.goff.push_back((int)p.gent.size());
      }
    }
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

// ------------------------------------------------------------------ level 1

LevelTopo build_level_one(int nx, int ny, int nz, int dpn, const uint8_t* dirichlet, const int32_t* elem_to_sub,
                          int n_subs, int initial, std::vector<int32_t>& elem_local) {
  const int64_t nnx = nx + 1, nny = ny + 1, nnz = nz + 1;
  const int64_t nn = nnx * nny * nnz;
  const int64_t nel = (int64_t)nx * ny * nz;
  LevelNodes N;
  N.n_dofs = nn * dpn;
  N.subs.assign(nn, {});
  N.tags.assign(nn, 0);
  N.eligible.assign(nn, 1);
  N.dofs.assign(nn, {});
  N.comps.assign(nn, {});
  for (int64_t e = 0; e < nel; ++e) {
    const int s = elem_to_sub[e];
    AMB_CHECK(s >= 0 && s < n_subs, AMB_EINVAL, "elem_to_sub out of range");
    const int64_t i = e % nx, j = (e / nx) % ny, k = e / ((int64_t)nx * ny);
    for (int a = 0; a < 8; ++a) {
      const int64_t n = (i + (a & 1)) + nnx * ((j + ((a >> 1) & 1)) + nny * (k + ((a >> 2) & 1)));
      auto& v = N.subs[n];
      if (std::find(v.begin(), v.end(), s) == v.end()) v.push_back(s);
    }
  }
  for (int64_t n = 0; n < nn; ++n) {
    std::sort(N.subs[n].begin(), N.subs[n].end());
    const int64_t i = n % nnx, j = (n / nnx) % nny, k = n / (nnx * nny);
    int t = 0;
    if (i == 0) t |= TAG_X0;
    if (i == nx) t |= TAG_X1;
    if (j == 0) t |= TAG_Y0;
    if (j == ny) t |= TAG_Y1;
    if (k == 0) t |= TAG_Z0;
    if (k == nz) t |= TAG_Z1;
    N.tags[n] = t;
    if (!dirichlet[n])
      for (int c = 0; c < dpn; ++c) {
        N.dofs[n].push_back(n * dpn + c);
        N.comps[n].push_back(c);
      }
  }
  LevelTopo L;
  L.n_subs = n_subs;
  classify(L, N, initial);
  L.node_tags_of_obj.clear();
  for (auto& ob : L.objs) L.node_tags_of_obj.push_back(ob.tags);
  number_coarse(L);
  // element -> local index in its substructure, -1 for Dirichlet dofs
  const int nd = 8 * dpn;
  elem_local.assign(nel * nd, -1);
  std::vector<int32_t> loc(nn * dpn, -1);
  std::vector<std::vector<int64_t>> elems_of(n_subs);
  for (int64_t e = 0; e < nel; ++e) elems_of[elem_to_sub[e]].push_back(e);
  for (int s = 0; s < n_subs; ++s) {
    const SubTopo& sb = L.subs[s];
    for (size_t q = 0; q < sb.dofs.size(); ++q) loc[sb.dofs[q]] = (int32_t)q;
    for (int64_t e : elems_of[s]) {
      const int64_t i = e % nx, j = (e / nx) % ny, k = e / ((int64_t)nx * ny);
      for (int a = 0; a < 8; ++a) {
        const int64_t n = (i + (a & 1)) + nnx * ((j + ((a >> 1) & 1)) + nny * (k + ((a >> 2) & 1)));
        for (int c = 0; c < dpn; ++c) {
          if (dirichlet[n]) continue;
          elem_local[e * nd + a * dpn + c] = loc[n * dpn + c];
        }
      }
    }
    for (size_t q = 0; q < sb.dofs.size(); ++q) loc[sb.dofs[q]] = -1;
  }
  return L;
}

// ------------------------------------------------------------------ level i+1

LevelTopo build_level_next(const LevelTopo& prev, const int32_t* parent, int n_subs, int initial,
                           std::vector<int32_t>& elem_local) {
  LevelNodes N;
  N.n_dofs = prev.n_coarse;
  const int no = (int)prev.objs.size();
  N.subs.assign(no, {});
  N.tags.assign(no, 0);
  N.eligible.assign(no, 0);
  N.dofs.assign(no, {});
  N.comps.assign(no, {});
  for (int o = 0; o < no; ++o) {
    const CoarseObj& ob = prev.objs[o];
    std::vector<int> ps;
    for (int s : ob.subs) {
      AMB_CHECK(parent[s] >= 0 && parent[s] < n_subs, AMB_EINVAL, "sub_to_parent out of range");
      ps.push_back(parent[s]);
    }
    std::sort(ps.begin(), ps.end());
    ps.erase(std::unique(ps.begin(), ps.end()), ps.end());
    N.subs[o] = ps;
    N.tags[o] = ob.tags;
    N.eligible[o] = ob.kind == OBJ_CORNER;
    for (size_t q = 0; q < ob.dofs.size(); ++q) {
      N.dofs[o].push_back(ob.first + (int64_t)q);
      N.comps[o].push_back(ob.comps[q]);
    }
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
