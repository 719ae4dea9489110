// waves.cu - the paper's cell-task schedule as a host tool (Sec. II.B and the Appendix).
//
// The paper runs the cell tasks of its CPU method (one task per grid cell) as a
// dependent task graph: tasks are grouped into "waves" of non-overlapping tasks
// (cells at least three apart in some dimension, so that their 3x3x3 neighbourhoods
// do not intersect), and every task waits only for the last earlier task that
// touched each of its cells.  This file builds
//   * the index sets that cover one dimension (Appendix),
//   * the waves of a 3-D grid by nested loops over those sets (Appendix),
//   * the dependent schedule by the forward or the backward wave method (Sec. II.B):
//     per task its number of direct predecessors and its list of direct successors,
// so that the paper's schedule can be checked against its own examples and compared
// with the 8 colour phases the GPU path uses.  Host code only; no device work.
//
// Reading of the Appendix used here.  In one dimension of D cells the index stream
// advances in steps of three (wrapping at D when periodic); the current set is closed
// when the next index would come closer than three cells to one of its members (the
// periodic distance when periodic) or when every cell is covered.  Without periodicity,
// or when D is a multiple of three, this gives the three residue classes.  When an
// outer loop advances, the inner dimension's stream restarts at the first index of
// its previous last set, so that consecutive waves differ by a shift in one direction
// (the Appendix's fifth wave, {9,12} filled to {9,12,1,4} for D = 14, follows).
// The 18-cell variant (Sec. II.D.3: tasks accessing a 3x3x2 block) spaces the z sets
// two cells apart.
#include "mdgb_waves.h"

#include <algorithm>
#include <cstring>
#include <vector>

namespace {

int cdist(int a, int b, int D, bool periodic) {
    int d = a > b ? a - b : b - a;
    if (periodic && D - d < d) d = D - d;
    return d;
}

// Ordered index sets covering 0..D-1 with members at least `spacing` apart, starting the
// stream at `start`.
std::vector<std::vector<int>> cover_1d(int D, bool periodic, int spacing, int start) {
    std::vector<std::vector<int>> sets;
    if (!periodic || D % spacing == 0) {
        // residue classes, beginning with the one holding `start`
        for (int k = 0; k < spacing && k < D; ++k) {
            const int r = (start + k) % spacing;
            std::vector<int> s;
            for (int x = r; x < D; x += spacing) s.push_back(x);
            if (!s.empty()) sets.push_back(s);
        }
        return sets;
    }
    std::vector<char> used(D, 0);
    int covered = 0, x = start % D;
    std::vector<int> cur;
    while (covered < D) {
        if (used[x]) {  // the stream came back to a covered cell: jump to the next free one
            int y = x;
            while (used[y]) y = (y + 1) % D;
            x = y;
        }
        bool clash = false;
        for (int m : cur)
            if (cdist(m, x, D, true) < spacing) clash = true;
        if (clash) {
            sets.push_back(cur);
            cur.clear();
        }
        cur.push_back(x);
        used[x] = 1;
        ++covered;
        x = (x + spacing) % D;
    }
    if (!cur.empty()) sets.push_back(cur);
    return sets;
}

struct Grid {
    int n[3];
    bool periodic[3];
    int overlap;  // 27 or 18
    int cell(int x, int y, int z) const { return x + n[0] * (y + n[1] * z); }
};

// Waves as lists of cells, in wave order (z outer, y middle, x inner).
std::vector<std::vector<int>> make_waves(const Grid& g) {
    const int sz = g.overlap == 18 ? 2 : 3;
    std::vector<std::vector<int>> waves;
    int ystart = 0, xstart = 0;
    for (const auto& zs : cover_1d(g.n[2], g.periodic[2], sz, 0)) {
        const auto ysets = cover_1d(g.n[1], g.periodic[1], 3, ystart);
        for (const auto& ys : ysets) {
            const auto xsets = cover_1d(g.n[0], g.periodic[0], 3, xstart);
            for (const auto& xs : xsets) {
                std::vector<int> w;
                for (int z : zs)
                    for (int y : ys)
                        for (int x : xs) w.push_back(g.cell(x, y, z));
                waves.push_back(w);
            }
            xstart = xsets.back().front();
        }
        ystart = ysets.back().front();
    }
    return waves;
}

// Cells a task at (x, y, z) touches: the 3x3x3 block around it, or the 3x3x2 block
// z..z+1 (18-cell variant); without periodicity, cells outside the grid are dropped.
void access_set(const Grid& g, int c, std::vector<int>& out) {
    out.clear();
    const int x = c % g.n[0], y = (c / g.n[0]) % g.n[1], z = c / (g.n[0] * g.n[1]);
    const int zlo = g.overlap == 18 ? 0 : -1;
    for (int dz = zlo; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                int p[3] = {x + dx, y + dy, z + dz};
                bool ok = true;
                for (int d = 0; d < 3; ++d) {
                    if (p[d] < 0 || p[d] >= g.n[d]) {
                        if (!g.periodic[d]) ok = false;
                        p[d] = (p[d] + g.n[d]) % g.n[d];
                    }
                }
                if (ok) out.push_back(g.cell(p[0], p[1], p[2]));
            }
    std::sort(out.begin(), out.end());
    out.erase(std::unique(out.begin(), out.end()), out.end());
}

bool make_grid(const int32_t n[3], const int32_t periodic[3], int32_t overlap, Grid& g) {
    if (!n || !periodic || (overlap != 27 && overlap != 18)) return false;
    for (int d = 0; d < 3; ++d) {
        if (n[d] < 1 || n[d] > 4096) return false;
        g.n[d] = n[d];
        g.periodic[d] = periodic[d] != 0;
        // a periodic dimension needs room for two non-overlapping tasks
        if (g.periodic[d] && n[d] < 3) return false;
    }
    if ((int64_t)n[0] * n[1] * n[2] > (1 << 28)) return false;
    g.overlap = overlap;
    return true;
}

}  // namespace

extern "C" {

int md_wave_sets_1d(int32_t D, int32_t periodic, int32_t spacing, int32_t start, int32_t* set_of_cell) {
    if (D < 1 || !set_of_cell || spacing < 1 || start < 0 || start >= D) return MD_ERR_ARG;
    if (periodic && D < spacing) return MD_ERR_ARG;
    const auto sets = cover_1d(D, periodic != 0, spacing, start);
    for (size_t k = 0; k < sets.size(); ++k)
        for (int x : sets[k]) set_of_cell[x] = (int32_t)k;
    return (int)sets.size();
}

int md_waves(const int32_t n[3], const int32_t periodic[3], int32_t overlap, int32_t* wave_of_cell) {
    Grid g;
    if (!make_grid(n, periodic, overlap, g) || !wave_of_cell) return MD_ERR_ARG;
    const auto waves = make_waves(g);
    for (size_t w = 0; w < waves.size(); ++w)
        for (int c : waves[w]) wave_of_cell[c] = (int32_t)w;
    return (int)waves.size();
}

int64_t md_wave_schedule(const int32_t n[3], const int32_t periodic[3], int32_t overlap, int32_t backward,
                         int32_t* task_cell, int32_t* n_pred, int64_t* succ_start, int32_t* succ, int64_t succ_cap) {
    Grid g;
    if (!make_grid(n, periodic, overlap, g) || !task_cell || !n_pred || !succ_start) return MD_ERR_ARG;
    const auto waves = make_waves(g);
    const int ncell = g.n[0] * g.n[1] * g.n[2];
    // tasks: one per cell, numbered in wave order
    std::vector<int> cell_of;
    cell_of.reserve(ncell);
    for (const auto& w : waves)
        for (int c : w) cell_of.push_back(c);
    if ((int)cell_of.size() != ncell) return MD_ERR_STATE;  // the waves must cover every cell once
    std::vector<std::vector<int>> succs(ncell);
    std::vector<int> npred(ncell, 0);
    std::vector<int> mark(ncell, -1);  // last (forward) or next (backward) task per cell
    std::vector<int> acc, lst;
    if (!backward) {
        // forward wave method: predecessors from the last task that accessed each cell
        for (int t = 0; t < ncell; ++t) {
            access_set(g, cell_of[t], acc);
            lst.clear();
            for (int c : acc)
                if (mark[c] >= 0) lst.push_back(mark[c]);
            std::sort(lst.begin(), lst.end());
            lst.erase(std::unique(lst.begin(), lst.end()), lst.end());
            npred[t] = (int)lst.size();
            for (int p : lst) succs[p].push_back(t);
            for (int c : acc) mark[c] = t;
        }
    } else {
        // backward wave method: successors from the next task that accesses each cell
        for (int t = ncell - 1; t >= 0; --t) {
            access_set(g, cell_of[t], acc);
            lst.clear();
            for (int c : acc)
                if (mark[c] >= 0) lst.push_back(mark[c]);
            std::sort(lst.begin(), lst.end());
            lst.erase(std::unique(lst.begin(), lst.end()), lst.end());
            succs[t] = lst;
            for (int s : lst) npred[s] += 1;
            for (int c : acc) mark[c] = t;
        }
    }
    int64_t total = 0;
    for (int t = 0; t < ncell; ++t) {
        std::sort(succs[t].begin(), succs[t].end());
        task_cell[t] = cell_of[t];
        n_pred[t] = npred[t];
        succ_start[t] = total;
        total += (int64_t)succs[t].size();
    }
    succ_start[ncell] = total;
    if (succ) {
        if (succ_cap < total) return MD_ERR_ARG;
        for (int t = 0; t < ncell; ++t)
            std::copy(succs[t].begin(), succs[t].end(), succ + succ_start[t]);
    }
    return total;
}

}  // extern "C"
