// Host mesh layer of the DOLINC library: validation, FP64 geometry (Sec 2.2),
// renumbering and the cell -> face slot tables the stage kernels read.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/dolinc.h"

namespace dol {

// Slot word: (internal face << 2) | (boundary << 1) | side, side 0 = the cell owns
// the face (area vector points out of it), side 1 = the cell is the neighbour.
inline uint32_t slot_word(int64_t f, bool bnd, int side) { return (uint32_t)((f << 2) | (bnd ? 2 : 0) | side); }

struct HostMesh {
    int dim = 0;
    int64_t n_cells = 0, n_faces = 0, n_bnd = 0, n_slots = 0;
    std::vector<int64_t> perm;          // new_of_old
    // FP64 geometry, library cell order
    std::vector<double> V, xc;          // [n_cells], [n_cells][3]
    // internal faces (owner = lower library index; sorted by owner, neighbour)
    std::vector<int64_t> fo, fn;        // owner / neighbour (-1 boundary)
    std::vector<double> fS, fxf, fd;    // [nf][3] area vector out of the internal owner, centroid, d
    std::vector<double> fw, fg;         // Eq 3 weight of the internal owner, Eq 4 growth rate
    std::vector<int64_t> face_ext;      // internal -> caller face
    std::vector<int8_t> face_flip;      // 1: internal orientation opposite to the caller's
    std::vector<int8_t> fkind;          // 0 interior, boundary: 1 zero-gradient, 2 Dirichlet, 3 Neumann
    // slots
    std::vector<int32_t> off;           // [n_cells+1]
    std::vector<int32_t> snb;           // neighbour cell of each slot (self on boundary)
    std::vector<uint32_t> sword;        // slot word
    std::vector<double> ss;             // [n_slots][3] (1-w_c) S_{c,f} / V_c
    std::vector<double> cw;             // [n_cells][4] (sum_f w_c S_{c,f} / V_c, 1/V_c)
    double g_min = 0, g_max = 0, h_min = 0, volume = 0;
    // skewness correction (empty: off): per cell M_c^-1 [n_cells][9], which the slot
    // and cell weights absorb; per internal face x_f - x*_f [n_faces][3]
    std::vector<double> minv, sdelta;
};

// Builds the host mesh; returns an empty string on success, else the error message.
std::string build_host_mesh(const dolinc_mesh_desc &d, HostMesh &m);

// Cell -> face slot tables (off, snb, sword, ss, cw) from the internal faces and the
// volumes: a cell's slots follow the internal face order.  With the skewness
// correction on, each cell's area vectors enter its weights as M_c^-1 S.
void build_slots(HostMesh &m);

// Turns the skewness correction on or off (minv, sdelta, then the slot tables).
// keep_identity (may be null): cells whose M_c^-1 is taken as the identity (ghost
// cells of a part, whose faces are not all present).  Returns an error message if
// some other cell's M_c is singular.
std::string apply_skew(HostMesh &m, bool on, const std::vector<uint8_t> *keep_identity);

// One part of a partition of a mesh (Sec 2.6: a coupled boundary exchanges only the
// adjacent cells' data and their differentials).  Local cells are the part's own
// cells and its ghosts (cells of other parts that share a face with an own cell),
// in the whole mesh's library order; local faces are the faces of the own cells, in
// the whole mesh's internal face order.  So every own cell sees the same faces, in
// the same order and orientation, with the same geometry as in the whole mesh.
struct PartPlan {
    int part = 0, n_parts = 0;
    std::vector<int64_t> cells;          // library index (whole mesh) of each local cell, ascending
    std::vector<uint8_t> owned;          // 1: an own cell, 0: a ghost
    std::vector<int64_t> faces;          // internal face index (whole mesh) of each local face, ascending
    std::vector<int32_t> peers;          // parts this part exchanges with, ascending
    // per peer (offsets into the lists, n_peers + 1): own cells the peer holds as
    // ghosts, and ghosts the peer owns; local indices, each list in ascending library
    // order, so a sender's list to q and q's list from the sender name the same cells
    // in the same order
    std::vector<int64_t> send_off, send_cells, recv_off, recv_cells;
};

// Plans part `part` of whole mesh g; part_lib[c] is the part of library cell c.
std::string plan_part(const HostMesh &g, const std::vector<int32_t> &part_lib, int n_parts, int part, PartPlan &p);

// The part's local host mesh: geometry and face tables copied from g, slots rebuilt.
void slice_host_mesh(const HostMesh &g, const PartPlan &p, HostMesh &out);

}  // namespace dol
