// Partition planning for halo-exchanged parts of one mesh (host side).
//
// A part holds its own cells and a depth-1 layer of ghost cells.  Each differential
// pass reads only face neighbours (Sec 2.3) and the face reconstruction only the two
// face cells' records (Sec 2.3-2.4), so the ghosts' records of every order the
// stage reads are all a part needs from its neighbours (Sec 2.6: coupled boundaries
// exchange the adjacent cells' data plus their differentials).
#include <algorithm>

#include "mesh.hpp"

namespace dol {

std::string plan_part(const HostMesh &g, const std::vector<int32_t> &part_lib, int n_parts, int part, PartPlan &p)
{
    const int64_t nc = g.n_cells, nf = g.n_faces;
    if (n_parts < 1) return "n_parts must be at least 1";
    if (part < 0 || part >= n_parts) return "part out of range";
    if ((int64_t)part_lib.size() != nc) return "one part per cell expected";
    for (int64_t c = 0; c < nc; ++c)
        if (part_lib[c] < 0 || part_lib[c] >= n_parts) return "part_of_cell entry out of range";
    p = PartPlan{};
    p.part = part;
    p.n_parts = n_parts;
    std::vector<uint8_t> local(nc, 0);      // 1 own, 2 ghost
    for (int64_t c = 0; c < nc; ++c)
        if (part_lib[c] == part) local[c] = 1;
    for (int64_t i = 0; i < nf; ++i) {
        const int64_t P = g.fo[i], N = g.fn[i];
        const bool own = local[P] == 1 || (N >= 0 && local[N] == 1);
        if (!own) continue;
        p.faces.push_back(i);
        if (N >= 0) {
            if (local[P] != 1) local[P] = 2;
            if (local[N] != 1) local[N] = 2;
        }
    }
    if (p.faces.empty()) return "the part owns no cell";
    std::vector<int64_t> loc(nc, -1);
    for (int64_t c = 0; c < nc; ++c)
        if (local[c]) {
            loc[c] = (int64_t)p.cells.size();
            p.cells.push_back(c);
            p.owned.push_back(local[c] == 1 ? 1 : 0);
        }
    // per peer: own cells adjacent to the peer's cells, and the peer's ghost cells
    std::vector<std::vector<int64_t>> snd(n_parts), rcv(n_parts);
    std::vector<int64_t> last_snd(n_parts, -1);
    for (size_t j = 0; j < p.cells.size(); ++j) {
        const int64_t c = p.cells[j];
        if (local[c] == 2) rcv[part_lib[c]].push_back((int64_t)j);
    }
    // own cell c is sent to every part that owns one of its face neighbours; the
    // cells are visited in ascending order, so each list comes out ascending
    std::vector<std::vector<int32_t>> adj(p.cells.size());
    for (int64_t i : p.faces) {
        const int64_t P = g.fo[i], N = g.fn[i];
        if (N < 0) continue;
        if (local[P] == 1 && local[N] == 2) adj[loc[P]].push_back(part_lib[N]);
        if (local[N] == 1 && local[P] == 2) adj[loc[N]].push_back(part_lib[P]);
    }
    for (size_t j = 0; j < p.cells.size(); ++j) {
        auto &a = adj[j];
        std::sort(a.begin(), a.end());
        a.erase(std::unique(a.begin(), a.end()), a.end());
        for (int32_t q : a) snd[q].push_back((int64_t)j);
    }
    p.send_off.push_back(0);
    p.recv_off.push_back(0);
    for (int q = 0; q < n_parts; ++q) {
        if (q == part || (snd[q].empty() && rcv[q].empty())) continue;
        p.peers.push_back(q);
        p.send_cells.insert(p.send_cells.end(), snd[q].begin(), snd[q].end());
        p.recv_cells.insert(p.recv_cells.end(), rcv[q].begin(), rcv[q].end());
        p.send_off.push_back((int64_t)p.send_cells.size());
        p.recv_off.push_back((int64_t)p.recv_cells.size());
    }
    return "";
}

void slice_host_mesh(const HostMesh &g, const PartPlan &p, HostMesh &m)
{
    const int64_t nc = (int64_t)p.cells.size(), nf = (int64_t)p.faces.size();
    std::vector<int64_t> loc(g.n_cells, -1);
    for (int64_t j = 0; j < nc; ++j) loc[p.cells[j]] = j;
    m = HostMesh{};
    m.dim = g.dim;
    m.n_cells = nc;
    m.n_faces = nf;
    m.perm.resize(nc);
    for (int64_t j = 0; j < nc; ++j) m.perm[j] = j;       // local caller order = local library order
    m.V.resize(nc);
    m.xc.resize(3 * nc);
    m.volume = 0;
    for (int64_t j = 0; j < nc; ++j) {
        const int64_t c = p.cells[j];
        m.V[j] = g.V[c];
        for (int k = 0; k < 3; ++k) m.xc[3 * j + k] = g.xc[3 * c + k];
        if (p.owned[j]) m.volume += g.V[c];
    }
    m.fo.resize(nf);
    m.fn.resize(nf);
    m.fS.resize(3 * nf);
    m.fxf.resize(3 * nf);
    m.fd.resize(3 * nf);
    m.fw.resize(nf);
    m.fg.resize(nf);
    m.face_ext.resize(nf);
    m.face_flip.assign(nf, 0);
    m.fkind.resize(nf);
    m.g_min = 1e300;
    m.g_max = 0;
    m.n_bnd = 0;
    for (int64_t k = 0; k < nf; ++k) {
        const int64_t i = p.faces[k];
        m.fo[k] = loc[g.fo[i]];
        m.fn[k] = g.fn[i] >= 0 ? loc[g.fn[i]] : -1;   // ascending local order: still the lower index
        for (int q = 0; q < 3; ++q) {
            m.fS[3 * k + q] = g.fS[3 * i + q];
            m.fxf[3 * k + q] = g.fxf[3 * i + q];
            m.fd[3 * k + q] = g.fd[3 * i + q];
        }
        m.fw[k] = g.fw[i];
        m.fg[k] = g.fg[i];
        m.face_ext[k] = k;                            // local caller faces = local internal faces
        m.fkind[k] = g.fkind[i];
        if (m.fn[k] < 0) {
            ++m.n_bnd;
        } else {
            m.g_min = std::min(m.g_min, std::min(m.fg[k], 1.0 / m.fg[k]));
            m.g_max = std::max(m.g_max, std::max(m.fg[k], 1.0 / m.fg[k]));
        }
    }
    if (m.g_max == 0) m.g_min = m.g_max = 1.0;
    build_slots(m);
    m.h_min = g.h_min;
}

}  // namespace dol
