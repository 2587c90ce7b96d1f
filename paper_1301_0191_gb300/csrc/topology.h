// Host-side substructuring of one decomposition level (Sec. 2, Sec. 3).
//
// Interface = nodes shared by >= 2 substructures; faces = nodes shared by
// the same two substructures; edges = nodes shared by the same set of more
// than two.  Corners are the vertices of the box grid (every coordinate on a
// cut plane or on the domain boundary), minus Dirichlet nodes.  The library
// sees only the element partition, so it uses the topological equivalent for
// box partitions: a node with b domain-boundary bits is a box vertex when
// 2^(3-b) substructures share it, and it must also be alone in its (sharing
// set, boundary bits) class.  "Alone in its class" by itself is not enough:
// next to a Dirichlet face a two-element segment leaves a face one node
// wide, whose node on the domain boundary is alone in its class but no
// vertex.  On level i >= 2 the nodes are the coarse objects of level i-1 and
// only level-(i-1) corners may become corners (under the same rule, with the
// level-i sharing sets).
#pragma once

#include <array>
#include <cstdint>
#include <vector>

namespace amb {

enum ObjKind { OBJ_CORNER = 0, OBJ_EDGE = 1, OBJ_ADAPTIVE = 2, OBJ_FACE = 3 };

// A coarse object: a corner node (one coarse dof per component), an edge or
// a face (one arithmetic average per component) or one adaptive face row.
struct CoarseObj {
  int kind = OBJ_CORNER;
  std::vector<int> subs;                      // sharing substructures (sorted)
  int tags = 0;                               // boundary-face bits common to its nodes
  std::vector<int> comps;                     // component of each coarse dof (-1 scalar)
  std::vector<std::vector<int64_t>> dofs;     // per coarse dof: level dofs of the functional
  std::vector<std::vector<double>> w;         // per coarse dof: weights
  int64_t first = 0;                          // global id of its first coarse dof
  int corner_node = -1;                       // level node id of a corner
};

struct SubTopo {
  std::vector<int64_t> dofs;                  // [interior | delta | corner] level dof ids
  int n_i = 0, n_g = 0, n_crn = 0;            // n_delta = n_g - n_crn
  std::vector<int64_t> rc;                    // global coarse ids: [corner dofs..., others...]
  // non-corner constraint rows on delta positions
  std::vector<std::vector<std::pair<int, double>>> crows;
  int n_c() const { return (int)rc.size(); }
  int n_d() const { return n_g - n_crn; }
  int n_cp() const { return n_c() - n_crn; }
};

struct PairTopo {
  int s = 0, t = 0;
  std::vector<int> ps, pt;                    // shared dof positions in the two interface blocks
  std::vector<int> face;                      // indices into ps/pt of face-class dofs
  std::vector<int64_t> face_dofs;             // their level dofs
  // jump constraints (initial coarse dofs shared by s and t): group g uses
  // entries [goff[g], goff[g+1]) of gent/gw (indices into ps/pt, weights)
  std::vector<int> goff, gent;
  std::vector<double> gw;
  // pair coarse space: union of the two substructures' coarse dofs
  int n_cpair = 0;
  std::vector<int> cmap_s, cmap_t;            // local coarse index -> pair coarse index
};

struct LevelTopo {
  int n_subs = 0;
  int64_t n_dofs = 0;
  std::vector<SubTopo> subs;
  std::vector<CoarseObj> objs;
  int64_t n_coarse = 0;
  int n_corner_nodes = 0, n_edges = 0, n_faces = 0;
  // global interface numbering and owners (CSR)
  std::vector<int64_t> iface_dofs;            // level dof of each global interface index
  std::vector<int> own_off;                   // size n_iface+1
  std::vector<int> own_sub, own_pos;          // owner substructure, position in its interface block
  std::vector<std::vector<int>> gidx;         // per sub: interface position -> global interface index
  std::vector<PairTopo> pairs;
  std::vector<int64_t> corner_dofs;           // level dofs of all corner dofs
  // nodes of this level (kept to build the next level's tags)
  std::vector<int> node_tags_of_obj;          // per object: common boundary bits
};

// Checks the decomposition hierarchy before anything is built: element and
// parent indices in range, no empty substructure, and every substructure of
// every level a box of elements (the box-vertex corner rule and the edge
// classes assume box partitions, Sec. 2 and 7.1).  parents[i] maps level-(i+1)
// substructures to level-(i+2) ones; nsubs[i] = substructures on level i+1.
// Throws Error(AMB_EINVAL) naming the first violation.  Host arrays only.
void validate_partition(int nx, int ny, int nz, const int32_t* elem_to_sub,
                        const std::vector<std::vector<int32_t>>& parents, const std::vector<int>& nsubs);

// Level 1 from the mesh.  dirichlet: per node; elem_to_sub: per element.
LevelTopo build_level_one(int nx, int ny, int nz, int dpn, const uint8_t* dirichlet, const int32_t* elem_to_sub,
                          int n_subs, int initial, std::vector<int32_t>& elem_local /* n_el * 8*dpn */);

// Level i+1 from level i and the parent map; elem_local receives, for each
// level-i substructure, the local index in its parent of each of its coarse dofs.
LevelTopo build_level_next(const LevelTopo& prev, const int32_t* parent, int n_subs, int initial,
                           std::vector<int32_t>& elem_local);

// Number coarse dofs, fill per-substructure rc/crows and the pair data, then
// check_topology.
void number_coarse(LevelTopo& L);

// Every index map the device kernels gather or scatter through is in range
// and consistent (interface numbering and owners, constraint positions, the
// pairs' shared positions, jump groups and coarse maps); throws
// Error(AMB_EINVAL, "internal topology check failed: ...") otherwise, so a
// fault in the host combinatorics stops the set-up before any kernel reads
// out of bounds.
void check_topology(const LevelTopo& L);

// Append adaptive rows (functionals on the face dofs of pair p).
void add_adaptive_rows(LevelTopo& L, int p, const std::vector<std::vector<double>>& rows);

}  // namespace amb
