// Device-resident mesh tables read by the stage kernels (all owned by the library).
#pragma once
#include <stdint.h>
#include <cuda_runtime.h>

namespace dol {

struct DevMesh {
    int dim, n_cells, n_faces, n_slots;
    const int32_t *off;          // [n_cells+1] slot ranges
    const int2 *slot2;           // [n_slots] (neighbour cell, slot word)
    const uint32_t *sword;       // [n_slots + 4] the slot words alone (16-byte aligned groups of 4)
    const double *slotk64;       // [n_slots][4] ((1-w_c) S_{c,f} / V_c, neighbour id bits)
    const float *slotk32;
    const double *cellk64;       // [n_cells][4] (sum_f w_c S_{c,f} / V_c, 1/V_c)
    const float *cellk32;
    const double *face64;        // [n_faces][8] (d, g, S, |S|), internal orientation
    const float *face32;
    const int32_t *fo, *fn;      // [n_faces] internal owner / neighbour (-1 boundary)
    const int32_t *face_ext;     // [n_faces] caller face id
    const int8_t *face_flip;     // [n_faces] 1 if the caller orientation is reversed
    const int32_t *fown;         // [n_cells+1] first internal face owned by each cell
    int max_tile_faces[3];       // most faces owned by a tile of 64 / 128 / 256 cells
    int max_slots;               // most slots of one cell
    int uniform_slots;           // slots of every cell when all cells have the same number, else 0
    // Dirichlet / Neumann boundary faces (Sec 2.6), n_bv of them
    int n_bv;
    const int32_t *bidx;         // [n_faces] index of the face among them, -1 otherwise (null: none)
    const int8_t *bkind;         // [n_bv] 2 Dirichlet, 3 Neumann
    const double *bdelta64;      // [n_bv] centroid-to-face distance along the outward unit normal
    const float *bdelta32;
    const double *bval64;        // [nv][n_bv] face value (Dirichlet) or outward normal gradient
    const float *bval32;         //   (Neumann), set by dolinc_set_boundary_values (null until then)
    int n_bcell;                 // cells with such faces, and their faces (CSR)
    const int32_t *bcell, *bcell_off, *bcell_face;
    // skewness correction (null: off): per internal face x_f - x*_f, padded to 4 values
    const double *fdelta64;
    const float *fdelta32;
};

}  // namespace dol
