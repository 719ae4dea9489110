// debug.cu - host-only introspection of the cell numbering (include/mdgb_debug.h).
#include "mdgb.h"
#include "mdgb_debug.h"
#include "tile.cuh"

#include <cmath>

using namespace mdgb;

namespace {

bool make_geometry(const int32_t nc[3], Geometry& g) {
    if (!nc) return false;
    for (int d = 0; d < 3; ++d) {
        if (nc[d] < 4 || nc[d] % 2 != 0 || nc[d] > 1024) return false;
        g.nc[d] = nc[d];
    }
    set_block_layout(g);
    return true;
}

}  // namespace

extern "C" {

int mdgb_grid_shape(const double box[3], double r_list, int32_t list_kind, int32_t nc_out[3]) {
    if (!box || !nc_out || !(r_list > 0.0) || list_kind < MD_LIST_FULL || list_kind > MD_LIST_HALF_ATOMIC_FREE)
        return MD_ERR_ARG;
    for (int d = 0; d < 3; ++d) {
        const int fit = (int)std::min(std::floor(box[d] / (r_list * (1.0 + 1e-12))), 1024.0);
        const int nc = grid_cells(fit, list_kind == MD_LIST_FULL);
        if (nc < 4) return MD_ERR_BOX_TOO_SMALL;
        nc_out[d] = nc;
    }
    return MD_OK;
}

int mdgb_coarse_cells(double side, double rho, double per_block, int32_t fit_nc, int32_t* nc_out) {
    if (!nc_out || !(side > 0.0) || !(rho > 0.0) || !(per_block > 0.0) || fit_nc < 4 || !std::isfinite(side) ||
        !std::isfinite(rho) || !std::isfinite(per_block))
        return MD_ERR_ARG;
    *nc_out = coarse_cells(side, rho, per_block, fit_nc);
    return MD_OK;
}

int mdgb_cut_band(int32_t frame, double w_max, double half_skin, int32_t R, double r_cut, double* band_out) {
    if (!band_out || !(w_max > 0.0) || !(half_skin >= 0.0) || !(r_cut > 0.0) || (frame != 0 && frame != 1) ||
        (frame == 1 && (R < 1 || R > 2)))
        return MD_ERR_ARG;
    *band_out = frame == 0 ? tile_frame_cut_band(w_max, half_skin, r_cut) : cell_frame_cut_band(w_max, R, r_cut);
    return MD_OK;
}

int mdgb_num_blocks(const int32_t nc[3], int32_t* nblock_out) {
    Geometry g{};
    if (!nblock_out || !make_geometry(nc, g)) return MD_ERR_ARG;
    *nblock_out = g.nblock;
    return MD_OK;
}

int mdgb_block_colour(const int32_t nc[3], int32_t block, int32_t* colour_out) {
    Geometry g{};
    if (!colour_out || !make_geometry(nc, g) || g.linear || block < 0 || block >= g.nblock) return MD_ERR_ARG;
    int bx, by, bz;
    block_coords(g, block, bx, by, bz);
    *colour_out = (bx & 1) | ((by & 1) << 1) | ((bz & 1) << 2);
    return MD_OK;
}

int mdgb_tile_cells(const int32_t nc[3], int32_t block, int32_t cells_out[64]) {
    Geometry g{};
    if (!cells_out || !make_geometry(nc, g) || block < 0 || block >= g.nblock) return MD_ERR_ARG;
    constexpr TileTables tt = make_tile_tables();
    int bx, by, bz;
    block_coords(g, block, bx, by, bz);
    for (int t = 0; t < 64; ++t) {
        const int c = tt.coord_of_idx[t];
        int cx = 2 * bx - 1 + (c & 3), cy = 2 * by - 1 + ((c >> 2) & 3), cz = 2 * bz - 1 + (c >> 4);
        cx = (cx + g.nc[0]) % g.nc[0];
        cy = (cy + g.nc[1]) % g.nc[1];
        cz = (cz + g.nc[2]) % g.nc[2];
        // round trip through the kernels' cell id to check the numbering is a bijection
        int id = cell_id_of(g, cx, cy, cz);
        int ax, ay, az;
        cell_coords(g, id, ax, ay, az);
        if (ax != cx || ay != cy || az != cz) return MD_ERR_ARG;
        cells_out[t] = cx + g.nc[0] * (cy + g.nc[1] * cz);
    }
    return MD_OK;
}

}  // extern "C"
