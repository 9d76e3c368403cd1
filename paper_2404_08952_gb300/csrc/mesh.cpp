// Host mesh layer: validation, FP64 geometry (Sec 2.2 Eqs 1-4), Morton renumbering
// and the cell -> face slot tables of the stage kernels.
//
// Geometry definition (shared with the ABI documentation): a 2D face a->b has area
// vector (b_y-a_y, -(b_x-a_x)) and centre (a+b)/2; a 3D triangle has area vector
// (b-a)x(c-a)/2 and centre (a+b+c)/3; a 3D polygon is the union of the triangles
// joining each edge to the mean of its nodes, with the sum of their area vectors and
// the area-weighted mean of their centres.  A cell is the polytope bounded by these
// pieces; volume and centroid are summed over the pyramids joining each piece to the
// mean of the cell's face centres.  A periodic face's neighbour side is the owner
// side translated by -shift.
#include "mesh.hpp"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <numeric>

namespace dol {

namespace {

struct V3 {
    double x = 0, y = 0, z = 0;
};
inline V3 operator+(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
inline V3 operator-(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
inline V3 operator*(double s, V3 a) { return {s * a.x, s * a.y, s * a.z}; }
inline double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline V3 cross(V3 a, V3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
inline double norm(V3 a) { return std::sqrt(dot(a, a)); }

std::string fmt(const char *f, long long a, long long b = 0)
{
    char buf[256];
    std::snprintf(buf, sizeof buf, f, a, b);
    return buf;
}

struct Piece {
    V3 S, c;
};

// area-vector pieces of face f (owner side)
void pieces(const dolinc_mesh_desc &d, int64_t f, std::vector<Piece> &out)
{
    out.clear();
    const int64_t o = d.face_node_offsets[f], n = d.face_node_offsets[f + 1] - o;
    auto P = [&](int64_t i) {
        const double *p = d.nodes + d.face_nodes[o + i] * d.dim;
        V3 v;
        v.x = p[0];
        v.y = p[1];
        v.z = d.dim == 3 ? p[2] : 0.0;
        return v;
    };
    if (d.dim == 2) {
        V3 a = P(0), b = P(1);
        out.push_back({V3{b.y - a.y, -(b.x - a.x), 0.0}, 0.5 * (a + b)});
        return;
    }
    if (n == 3) {
        V3 a = P(0), b = P(1), c = P(2);
        out.push_back({0.5 * cross(b - a, c - a), (1.0 / 3.0) * (a + b + c)});
        return;
    }
    V3 mc;
    for (int64_t i = 0; i < n; ++i) mc = mc + P(i);
    mc = (1.0 / (double)n) * mc;
    for (int64_t i = 0; i < n; ++i) {
        V3 a = P(i), b = P((i + 1) % n);
        out.push_back({0.5 * cross(a - mc, b - mc), (1.0 / 3.0) * (mc + a + b)});
    }
}

uint64_t spread3(uint64_t v)   // 21 bits -> every third bit
{
    v &= 0x1fffff;
    v = (v | v << 32) & 0x1f00000000ffffULL;
    v = (v | v << 16) & 0x1f0000ff0000ffULL;
    v = (v | v << 8) & 0x100f00f00f00f00fULL;
    v = (v | v << 4) & 0x10c30c30c30c30c3ULL;
    v = (v | v << 2) & 0x1249249249249249ULL;
    return v;
}
uint64_t spread2(uint64_t v)   // 31 bits -> every second bit
{
    v &= 0x7fffffff;
    v = (v | v << 16) & 0x0000ffff0000ffffULL;
    v = (v | v << 8) & 0x00ff00ff00ff00ffULL;
    v = (v | v << 4) & 0x0f0f0f0f0f0f0f0fULL;
    v = (v | v << 2) & 0x3333333333333333ULL;
    v = (v | v << 1) & 0x5555555555555555ULL;
    return v;
}

}  // namespace

// Cell -> face slot tables from the internal faces (fo, fn, fS, fw) and volumes:
// a cell's slots follow the internal face order.
void build_slots(HostMesh &m)
{
    const int64_t nc = m.n_cells, nf = m.n_faces;
    m.off.assign(nc + 1, 0);
    for (int64_t i = 0; i < nf; ++i) {
        m.off[m.fo[i] + 1]++;
        if (m.fn[i] >= 0) m.off[m.fn[i] + 1]++;
    }
    for (int64_t c = 0; c < nc; ++c) m.off[c + 1] += m.off[c];
    m.n_slots = m.off[nc];
    m.snb.resize(m.n_slots);
    m.sword.resize(m.n_slots);
    m.ss.assign(3 * m.n_slots, 0.0);
    m.cw.assign(4 * nc, 0.0);
    std::vector<int32_t> fill(m.off.begin(), m.off.end() - 1);
    // slots of a cell follow the internal face order
    const bool skew = !m.minv.empty();
    // M_c^-1 S (skewness correction) or S
    auto corr = [&](int64_t c, V3 s) {
        if (!skew) return s;
        const double *a = &m.minv[9 * c];
        return V3{a[0] * s.x + a[1] * s.y + a[2] * s.z, a[3] * s.x + a[4] * s.y + a[5] * s.z,
                  a[6] * s.x + a[7] * s.y + a[8] * s.z};
    };
    for (int64_t i = 0; i < nf; ++i) {
        const int64_t P = m.fo[i], N = m.fn[i];
        const V3 s0{m.fS[3 * i], m.fS[3 * i + 1], m.fS[3 * i + 2]};
        const double w = m.fw[i];
        {
            const V3 s = corr(P, s0);
            int64_t sl = fill[P]++;
            m.snb[sl] = (int32_t)(N >= 0 ? N : P);
            m.sword[sl] = slot_word(i, N < 0, 0);
            double iv = 1.0 / m.V[P];
            // weight of P at the face: w (boundary: w = 1, face value = cell value)
            V3 k = ((1.0 - w) * iv) * s;
            m.ss[3 * sl] = k.x, m.ss[3 * sl + 1] = k.y, m.ss[3 * sl + 2] = k.z;
            m.cw[4 * P] += w * iv * s.x, m.cw[4 * P + 1] += w * iv * s.y, m.cw[4 * P + 2] += w * iv * s.z;
        }
        if (N >= 0) {
            const V3 s = corr(N, s0);
            int64_t sl = fill[N]++;
            m.snb[sl] = (int32_t)P;
            m.sword[sl] = slot_word(i, false, 1);
            double iv = 1.0 / m.V[N];
            // N sees -S with weight 1-w; its neighbour P gets weight w
            V3 k = (-w * iv) * s;
            m.ss[3 * sl] = k.x, m.ss[3 * sl + 1] = k.y, m.ss[3 * sl + 2] = k.z;
            double wn = (1.0 - w) * iv;
            m.cw[4 * N] -= wn * s.x, m.cw[4 * N + 1] -= wn * s.y, m.cw[4 * N + 2] -= wn * s.z;
        }
    }
    for (int64_t c = 0; c < nc; ++c) m.cw[4 * c + 3] = 1.0 / m.V[c];
}

std::string apply_skew(HostMesh &m, bool on, const std::vector<uint8_t> *keep_identity)
{
    const int64_t nc = m.n_cells, nf = m.n_faces;
    if (!on) {
        m.minv.clear();
        m.sdelta.clear();
        build_slots(m);
        return "";
    }
    // M_c = (1/V_c) sum_f S_{c,f} (x) (x*_f - x_c): from the owner x*_f - x_P = (1-w) d,
    // from the neighbour (its own frame) x*_f - x_N = -w d; boundary faces x*_f = x_f
    std::vector<double> M(9 * nc, 0.0), sd(3 * nf, 0.0);
    for (int64_t i = 0; i < nf; ++i) {
        const int64_t P = m.fo[i], N = m.fn[i];
        const V3 s{m.fS[3 * i], m.fS[3 * i + 1], m.fS[3 * i + 2]};
        const V3 xf{m.fxf[3 * i], m.fxf[3 * i + 1], m.fxf[3 * i + 2]};
        const V3 xP{m.xc[3 * P], m.xc[3 * P + 1], m.xc[3 * P + 2]};
        const V3 dd{m.fd[3 * i], m.fd[3 * i + 1], m.fd[3 * i + 2]};
        const double w = m.fw[i];
        const V3 rP = N >= 0 ? (1.0 - w) * dd : xf - xP;
        const double sv[3] = {s.x, s.y, s.z}, rp[3] = {rP.x, rP.y, rP.z};
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) M[9 * P + 3 * a + b] += sv[a] * rp[b] / m.V[P];
        if (N >= 0) {
            const double rn[3] = {-w * dd.x, -w * dd.y, -w * dd.z};
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) M[9 * N + 3 * a + b] -= sv[a] * rn[b] / m.V[N];
            const V3 del = xf - (xP + rP);
            sd[3 * i] = del.x, sd[3 * i + 1] = del.y, sd[3 * i + 2] = del.z;
        }
    }
    std::vector<double> inv(9 * nc);
    for (int64_t c = 0; c < nc; ++c) {
        double *a = &M[9 * c], *b = &inv[9 * c];
        if (m.dim == 2) a[2] = a[5] = a[6] = a[7] = 0.0, a[8] = 1.0;
        const double det = a[0] * (a[4] * a[8] - a[5] * a[7]) - a[1] * (a[3] * a[8] - a[5] * a[6]) +
                           a[2] * (a[3] * a[7] - a[4] * a[6]);
        if ((keep_identity && (*keep_identity)[c]) || !(std::fabs(det) > 1e-12)) {
            if (!(keep_identity && (*keep_identity)[c]))
                return fmt("cell %lld: singular skewness matrix", c);
            for (int k = 0; k < 9; ++k) b[k] = (k % 4 == 0) ? 1.0 : 0.0;
            continue;
        }
        b[0] = (a[4] * a[8] - a[5] * a[7]) / det, b[1] = (a[2] * a[7] - a[1] * a[8]) / det;
        b[2] = (a[1] * a[5] - a[2] * a[4]) / det, b[3] = (a[5] * a[6] - a[3] * a[8]) / det;
        b[4] = (a[0] * a[8] - a[2] * a[6]) / det, b[5] = (a[2] * a[3] - a[0] * a[5]) / det;
        b[6] = (a[3] * a[7] - a[4] * a[6]) / det, b[7] = (a[1] * a[6] - a[0] * a[7]) / det;
        b[8] = (a[0] * a[4] - a[1] * a[3]) / det;
    }
    m.minv.swap(inv);
    m.sdelta.swap(sd);
    build_slots(m);
    return "";
}

std::string build_host_mesh(const dolinc_mesh_desc &d, HostMesh &m)
{
    // ---------------------------------------------------------------- validation
    if (d.dim != 2 && d.dim != 3) return "dim must be 2 or 3";
    if (d.n_nodes <= 0 || d.n_cells <= 0 || d.n_faces <= 0) return "empty mesh";
    if (!d.nodes || !d.face_node_offsets || !d.face_nodes || !d.face_owner || !d.face_neighbour)
        return "null mesh array";
    if (d.n_cells > (int64_t)1 << 30) return "too many cells (limit 2^30)";
    if (d.n_faces > (int64_t)1 << 29) return "too many faces (limit 2^29)";
    if (d.renumber != DOLINC_RENUMBER_NONE && d.renumber != DOLINC_RENUMBER_MORTON) return "unknown renumber mode";
    const int D = d.dim;
    const int64_t nc = d.n_cells, nf = d.n_faces;
    if (d.face_node_offsets[0] != 0) return "face_node_offsets[0] != 0";
    std::vector<int> nslot(nc, 0);
    int64_t nb = 0;
    for (int64_t f = 0; f < nf; ++f) {
        int64_t a = d.face_node_offsets[f], b = d.face_node_offsets[f + 1];
        if (b < a) return fmt("face %lld: decreasing node offsets", f);
        if (D == 2 && b - a != 2) return fmt("face %lld: a 2D face has 2 nodes, got %lld", f, b - a);
        if (D == 3 && (b - a < 3 || b - a > 64)) return fmt("face %lld: a 3D face has 3..64 nodes, got %lld", f, b - a);
        for (int64_t i = a; i < b; ++i)
            if (d.face_nodes[i] < 0 || d.face_nodes[i] >= d.n_nodes) return fmt("face %lld: node id out of range", f);
        int64_t P = d.face_owner[f], N = d.face_neighbour[f];
        if (P < 0 || P >= nc) return fmt("face %lld: owner %lld out of range", f, P);
        if (N < -1 || N >= nc) return fmt("face %lld: neighbour %lld out of range", f, N);
        if (N < 0) {
            ++nb;
            if (d.boundary_kind && (d.boundary_kind[f] < 1 || d.boundary_kind[f] > 3))
                return fmt("face %lld: boundary kind %lld unsupported (1 zero-gradient, 2 Dirichlet, 3 Neumann)", f,
                           (long long)d.boundary_kind[f]);
        } else if (d.boundary_kind && d.boundary_kind[f] != 0) {
            return fmt("face %lld: interior face with boundary kind %lld", f, (long long)d.boundary_kind[f]);
        }
        nslot[P]++;
        if (N >= 0) nslot[N]++;
    }
    for (int64_t c = 0; c < nc; ++c)
        if (nslot[c] < D + 1) return fmt("cell %lld has %lld faces (fewer than dim+1)", c, nslot[c]);
    if (d.cell_face_offsets && d.cell_faces) {
        if (d.cell_face_offsets[0] != 0) return "cell_face_offsets[0] != 0";
        for (int64_t c = 0; c < nc; ++c) {
            int64_t a = d.cell_face_offsets[c], b = d.cell_face_offsets[c + 1];
            if (b - a != nslot[c]) return fmt("cell %lld: cell_faces lists a different number of faces", c);
            for (int64_t i = a; i < b; ++i) {
                int64_t f = d.cell_faces[i];
                if (f < 0 || f >= nf || (d.face_owner[f] != c && d.face_neighbour[f] != c))
                    return fmt("cell %lld: cell_faces names a face that is not its own (%lld)", c, f);
            }
        }
    }
    m.dim = D;
    m.n_cells = nc;
    m.n_faces = nf;
    m.n_bnd = nb;

    // ---------------------------------------------------------------- geometry, caller order
    std::vector<V3> S(nf), xf(nf), sh(nf), apex(nc);
    std::vector<double> cnt(nc, 0.0);
    std::vector<Piece> pc;
    for (int64_t f = 0; f < nf; ++f) {
        pieces(d, f, pc);
        V3 s, c;
        double area = 0;
        for (auto &p : pc) {
            double a = norm(p.S);
            s = s + p.S;
            c = c + a * p.c;
            area += a;
        }
        if (!(area > 0)) return fmt("face %lld has zero area", f);
        S[f] = s;
        xf[f] = (1.0 / area) * c;
        if (d.face_periodic_shift && d.face_neighbour[f] >= 0) {
            const double *q = d.face_periodic_shift + f * D;
            sh[f] = V3{q[0], q[1], D == 3 ? q[2] : 0.0};
        }
        int64_t P = d.face_owner[f], N = d.face_neighbour[f];
        apex[P] = apex[P] + xf[f];
        cnt[P] += 1;
        if (N >= 0) {
            apex[N] = apex[N] + (xf[f] - sh[f]);
            cnt[N] += 1;
        }
    }
    for (int64_t c = 0; c < nc; ++c) apex[c] = (1.0 / cnt[c]) * apex[c];
    std::vector<double> V(nc, 0.0);
    std::vector<V3> mom(nc), close(nc);
    std::vector<double> amax(nc, 0.0);
    for (int64_t f = 0; f < nf; ++f) {
        pieces(d, f, pc);
        int64_t P = d.face_owner[f], N = d.face_neighbour[f];
        for (int side = 0; side < (N >= 0 ? 2 : 1); ++side) {
            int64_t c = side ? N : P;
            double sg = side ? -1.0 : 1.0;
            V3 off = side ? sh[f] : V3{};
            for (auto &p : pc) {
                V3 cc = p.c - off;
                double vol = sg * dot(p.S, cc - apex[c]) / (double)D;
                V[c] += vol;
                mom[c] = mom[c] + (vol / (double)(D + 1)) * (apex[c] + (double)D * cc);
            }
            close[c] = close[c] + sg * S[f];
            amax[c] = std::max(amax[c], norm(S[f]));
        }
    }
    // ---------------------------------------------------------------- renumbering
    std::vector<V3> xcold(nc);
    double vtot = 0;
    for (int64_t c = 0; c < nc; ++c) {
        if (!(V[c] > 0)) return fmt("cell %lld has non-positive volume", c);
        if (norm(close[c]) > 1e-9 * amax[c] * cnt[c]) return fmt("cell %lld is not closed (check face orientation)", c);
        xcold[c] = (1.0 / V[c]) * mom[c];
        vtot += V[c];
    }
    m.volume = vtot;
    m.perm.resize(nc);
    if (d.renumber == DOLINC_RENUMBER_MORTON) {
        V3 lo = xcold[0], hi = xcold[0];
        for (auto &x : xcold) {
            lo = V3{std::min(lo.x, x.x), std::min(lo.y, x.y), std::min(lo.z, x.z)};
            hi = V3{std::max(hi.x, x.x), std::max(hi.y, x.y), std::max(hi.z, x.z)};
        }
        std::vector<std::pair<uint64_t, int64_t>> key(nc);
        const double bits = D == 3 ? 2097151.0 : 2147483647.0;
        for (int64_t c = 0; c < nc; ++c) {
            auto q = [&](double v, double a, double b) { return (uint64_t)(b > a ? (v - a) / (b - a) * bits : 0.0); };
            uint64_t ix = q(xcold[c].x, lo.x, hi.x), iy = q(xcold[c].y, lo.y, hi.y), iz = q(xcold[c].z, lo.z, hi.z);
            uint64_t k = D == 3 ? (spread3(ix) | spread3(iy) << 1 | spread3(iz) << 2) : (spread2(ix) | spread2(iy) << 1);
            key[c] = {k, c};
        }
        std::sort(key.begin(), key.end());
        for (int64_t i = 0; i < nc; ++i) m.perm[key[i].second] = i;
    } else {
        std::iota(m.perm.begin(), m.perm.end(), (int64_t)0);
    }
    m.V.assign(nc, 0.0);
    m.xc.assign(3 * nc, 0.0);
    for (int64_t c = 0; c < nc; ++c) {
        int64_t n = m.perm[c];
        m.V[n] = V[c];
        m.xc[3 * n] = xcold[c].x;
        m.xc[3 * n + 1] = xcold[c].y;
        m.xc[3 * n + 2] = xcold[c].z;
    }
    // ---------------------------------------------------------------- internal faces
    struct FK {
        int64_t o, n, f;
        bool flip;
    };
    std::vector<FK> fk(nf);
    for (int64_t f = 0; f < nf; ++f) {
        int64_t P = m.perm[d.face_owner[f]];
        int64_t N = d.face_neighbour[f] >= 0 ? m.perm[d.face_neighbour[f]] : -1;
        bool flip = N >= 0 && N < P;
        fk[f] = flip ? FK{N, P, f, true} : FK{P, N, f, false};
    }
    std::sort(fk.begin(), fk.end(), [](const FK &a, const FK &b) {
        if (a.o != b.o) return a.o < b.o;
        int64_t an = a.n < 0 ? INT64_MAX : a.n, bn = b.n < 0 ? INT64_MAX : b.n;
        if (an != bn) return an < bn;
        return a.f < b.f;
    });
    m.fo.resize(nf);
    m.fn.resize(nf);
    m.fS.resize(3 * nf);
    m.fxf.resize(3 * nf);
    m.fd.resize(3 * nf);
    m.fw.resize(nf);
    m.fg.resize(nf);
    m.face_ext.resize(nf);
    m.face_flip.resize(nf);
    m.fkind.assign(nf, 0);
    m.g_min = 1e300;
    m.g_max = 0;
    for (int64_t i = 0; i < nf; ++i) {
        const FK &k = fk[i];
        const int64_t f = k.f;
        m.fo[i] = k.o;
        m.fn[i] = k.n;
        m.face_ext[i] = f;
        m.face_flip[i] = k.flip ? 1 : 0;
        if (k.n < 0) m.fkind[i] = (int8_t)(d.boundary_kind ? d.boundary_kind[f] : 1);
        // caller-orientation quantities first
        V3 s = S[f], x = xf[f];
        V3 xP = xcold[d.face_owner[f]];
        double w, g;
        V3 dd;
        if (k.n < 0) {
            w = 1.0;
            g = 1.0;
            dd = 2.0 * (x - xP);
        } else {
            V3 xN = xcold[d.face_neighbour[f]] + sh[f];
            double aN = norm(xN - x), aP = norm(x - xP);
            if (!(aN > 0) || !(aP > 0)) return fmt("face %lld: a cell centroid lies on the face", f);
            w = aN / (aP + aN);                 // Eq 3: weight of the owner
            g = aN / aP;                        // Eq 4
            dd = xN - xP;                       // Eq 2 (periodic translation included)
        }
        if (k.flip) {
            // internal owner is the caller's neighbour: its face centre is x - shift
            x = x - sh[f];
            s = -1.0 * s;
            w = 1.0 - w;
            g = 1.0 / g;
            dd = -1.0 * dd;
        }
        m.fS[3 * i] = s.x, m.fS[3 * i + 1] = s.y, m.fS[3 * i + 2] = s.z;
        m.fxf[3 * i] = x.x, m.fxf[3 * i + 1] = x.y, m.fxf[3 * i + 2] = x.z;
        m.fd[3 * i] = dd.x, m.fd[3 * i + 1] = dd.y, m.fd[3 * i + 2] = dd.z;
        m.fw[i] = w;
        m.fg[i] = g;
        if (k.n >= 0) {
            m.g_min = std::min(m.g_min, std::min(g, 1.0 / g));
            m.g_max = std::max(m.g_max, std::max(g, 1.0 / g));
        }
    }
    if (m.g_max == 0) m.g_min = m.g_max = 1.0;
    build_slots(m);
    m.h_min = 1e300;
    for (int64_t c = 0; c < nc; ++c) m.h_min = std::min(m.h_min, V[c] / std::max(amax[c], 1e-300));
    return "";
}

}  // namespace dol
