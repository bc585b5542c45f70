// swdg_forest.cu -- quadtree forests for dynamic h-adaptation (Sec. 3.4):
// the refine/coarsen criteria, the smallest 2:1-balanced leaf set after
// refinement and coarsening, the Morton order of the leaves and the mesh
// (geometry and neighbour slots of the C-ABI) of a leaf set.  Host code only.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <unordered_set>
#include <unordered_map>
#include <vector>

#include "../../include/swdg.h"
#include "swdg_forest.h"

namespace swdg {

static inline uint64_t pack(int l, int64_t i, int64_t j) {
    return ((uint64_t)l << 58) | ((uint64_t)i << 29) | (uint64_t)j;
}

bool Forest::wrap(int l, int64_t i, int64_t j, int64_t& ii, int64_t& jj) const {
    const int64_t nxl = (int64_t)f.nx0 << l, nyl = (int64_t)f.ny0 << l;
    if (f.periodic[0]) i = ((i % nxl) + nxl) % nxl;
    if (f.periodic[1]) j = ((j % nyl) + nyl) % nyl;
    if (i < 0 || i >= nxl || j < 0 || j >= nyl) return false;
    ii = i;
    jj = j;
    return true;
}

// the leaf covering cell (l, i, j) if it is that cell or an ancestor
static bool covering(const std::unordered_set<uint64_t>& S, int l, int64_t i, int64_t j, Leaf* out) {
    while (l >= 0) {
        if (S.count(pack(l, i, j))) {
            if (out) *out = Leaf{l, (int32_t)i, (int32_t)j};
            return true;
        }
        --l;
        i >>= 1;
        j >>= 1;
    }
    return false;
}

// the two level-(l+1) cells of cell (l, ii, jj) along its face toward a
// neighbour in direction (di, dj), by increasing tangential coordinate
static void along(int l, int64_t ii, int64_t jj, int di, int dj, uint64_t out[2]) {
    if (di != 0) {
        const int a = di > 0 ? 0 : 1;
        out[0] = pack(l + 1, 2 * ii + a, 2 * jj);
        out[1] = pack(l + 1, 2 * ii + a, 2 * jj + 1);
    } else {
        const int b = dj > 0 ? 0 : 1;
        out[0] = pack(l + 1, 2 * ii, 2 * jj + b);
        out[1] = pack(l + 1, 2 * ii + 1, 2 * jj + b);
    }
}

static const int DIR[4][2] = {{-1, 0}, {1, 0}, {0, -1}, {0, 1}};

void Forest::flags(const std::vector<Leaf>& leaves, const double* eta, double theta_r,
                   double theta_c, int8_t* out) const {
    double emax = 0.0;
    for (size_t k = 0; k < leaves.size(); ++k) emax = std::max(emax, eta[k]);
    for (size_t k = 0; k < leaves.size(); ++k) {
        const int l = leaves[k].l;
        const double hx = f.hx0 / (double)(1 << l), hy = f.hy0 / (double)(1 << l);
        if (eta[k] > theta_r * emax && l < f.max_level && std::max(hx, hy) > f.h_min) out[k] = 1;
        else if (eta[k] < theta_c * emax && l > 0) out[k] = -1;
        else out[k] = 0;
    }
}

std::vector<Leaf> Forest::adapt(const std::vector<Leaf>& leaves, const int8_t* fl) const {
    std::unordered_set<uint64_t> S, marked;
    S.reserve(leaves.size() * 2);
    for (size_t k = 0; k < leaves.size(); ++k) {
        const Leaf c = leaves[k];
        if (fl[k] == 1) {
            for (int b = 0; b < 2; ++b)
                for (int a = 0; a < 2; ++a) S.insert(pack(c.l + 1, 2 * c.i + a, 2 * c.j + b));
        } else {
            S.insert(pack(c.l, c.i, c.j));
        }
        if (fl[k] == -1) marked.insert(pack(c.l, c.i, c.j));
    }
    // four siblings, all leaves and all marked, merge into their parent
    std::vector<uint64_t> done;
    for (size_t k = 0; k < leaves.size(); ++k) {
        if (fl[k] != -1) continue;
        const Leaf c = leaves[k];
        const int l = c.l - 1;
        const int64_t pi = c.i >> 1, pj = c.j >> 1;
        const uint64_t pk = pack(l, pi, pj);
        if (std::find(done.begin(), done.end(), pk) != done.end()) continue;
        done.push_back(pk);
        bool all = true;
        for (int b = 0; b < 2 && all; ++b)
            for (int a = 0; a < 2 && all; ++a) {
                const uint64_t ck = pack(l + 1, 2 * pi + a, 2 * pj + b);
                all = S.count(ck) && marked.count(ck);
            }
        if (!all) continue;
        for (int b = 0; b < 2; ++b)
            for (int a = 0; a < 2; ++a) S.erase(pack(l + 1, 2 * pi + a, 2 * pj + b));
        S.insert(pk);
    }
    // 2:1 balance: split every leaf whose face neighbour region holds leaves
    // two or more levels finer, until none does
    bool changed = true;
    while (changed) {
        changed = false;
        std::vector<uint64_t> cur(S.begin(), S.end());
        for (uint64_t key : cur) {
            if (!S.count(key)) continue;
            const int l = (int)(key >> 58);
            const int64_t i = (int64_t)((key >> 29) & ((1ull << 29) - 1)), j = (int64_t)(key & ((1ull << 29) - 1));
            for (int d = 0; d < 4; ++d) {
                int64_t ii, jj;
                if (!wrap(l, i + DIR[d][0], j + DIR[d][1], ii, jj)) continue;
                if (covering(S, l, ii, jj, nullptr)) continue;
                uint64_t al[2];
                along(l, ii, jj, DIR[d][0], DIR[d][1], al);
                if (S.count(al[0]) && S.count(al[1])) continue;
                S.erase(key);
                for (int b = 0; b < 2; ++b)
                    for (int a = 0; a < 2; ++a) S.insert(pack(l + 1, 2 * i + a, 2 * j + b));
                changed = true;
                break;
            }
        }
    }
    std::vector<Leaf> out;
    out.reserve(S.size());
    for (uint64_t key : S)
        out.push_back(Leaf{(int)(key >> 58), (int32_t)((key >> 29) & ((1ull << 29) - 1)),
                           (int32_t)(key & ((1ull << 29) - 1))});
    order(out);
    return out;
}

// Morton key of the lower-left corner on the grid of level max_level
uint64_t Forest::morton(const Leaf& c) const {
    const uint64_t x = (uint64_t)c.i << (f.max_level - c.l), y = (uint64_t)c.j << (f.max_level - c.l);
    uint64_t k = 0;
    for (int bit = 0; bit < 30; ++bit)
        k |= (((x >> bit) & 1ull) << (2 * bit)) | (((y >> bit) & 1ull) << (2 * bit + 1));
    return k;
}

void Forest::order(std::vector<Leaf>& leaves) const {
    std::sort(leaves.begin(), leaves.end(),
              [&](const Leaf& a, const Leaf& b) { return morton(a) < morton(b); });
}

void Forest::mesh(const std::vector<Leaf>& leaves, double* x0y0, double* hxhy, int32_t* nbr) const {
    std::unordered_map<uint64_t, int32_t> index;
    index.reserve(leaves.size() * 2);
    for (size_t k = 0; k < leaves.size(); ++k)
        index[pack(leaves[k].l, leaves[k].i, leaves[k].j)] = (int32_t)k;
    for (size_t k = 0; k < leaves.size(); ++k) {
        const Leaf c = leaves[k];
        const double hx = f.hx0 / (double)(1 << c.l), hy = f.hy0 / (double)(1 << c.l);
        x0y0[2 * k] = f.x0 + c.i * hx;
        x0y0[2 * k + 1] = f.y0 + c.j * hy;
        hxhy[2 * k] = hx;
        hxhy[2 * k + 1] = hy;
        for (int d = 0; d < 4; ++d) {
            int32_t* s = nbr + k * 8 + 2 * d;
            s[1] = -1;
            int64_t ii, jj;
            if (!wrap(c.l, (int64_t)c.i + DIR[d][0], (int64_t)c.j + DIR[d][1], ii, jj)) {
                s[0] = -1 - f.tags[d];
                continue;
            }
            auto it = index.find(pack(c.l, ii, jj));
            if (it != index.end()) {
                s[0] = it->second;
                continue;
            }
            if (c.l > 0) {
                it = index.find(pack(c.l - 1, ii >> 1, jj >> 1));
                if (it != index.end()) {
                    s[0] = it->second;
                    continue;
                }
            }
            uint64_t al[2];
            along(c.l, ii, jj, DIR[d][0], DIR[d][1], al);
            s[0] = index.at(al[0]);
            s[1] = index.at(al[1]);
        }
    }
}

// leaves of a mesh on this forest; false if a cell is not a leaf of it
bool Forest::leaves_of(int64_t n, const double* x0y0, const double* hxhy,
                       std::vector<Leaf>& out) const {
    out.resize(n);
    for (int64_t k = 0; k < n; ++k) {
        const double r = f.hx0 / hxhy[2 * k];
        const int l = (int)std::lround(std::log2(r));
        if (l < 0 || l > f.max_level || std::fabs(r - (double)(1 << l)) > 1e-9 * r ||
            std::fabs(f.hy0 / hxhy[2 * k + 1] - (double)(1 << l)) > 1e-9 * r)
            return false;
        const double hx = f.hx0 / (double)(1 << l), hy = f.hy0 / (double)(1 << l);
        const double fi = (x0y0[2 * k] - f.x0) / hx, fj = (x0y0[2 * k + 1] - f.y0) / hy;
        const int64_t i = std::llround(fi), j = std::llround(fj);
        if (std::fabs(fi - i) > 1e-6 || std::fabs(fj - j) > 1e-6 || i < 0 || j < 0 ||
            i >= ((int64_t)f.nx0 << l) || j >= ((int64_t)f.ny0 << l))
            return false;
        out[k] = Leaf{l, (int32_t)i, (int32_t)j};
    }
    return true;
}

bool forest_valid(const swdg_forest* f) {
    return f && f->nx0 > 0 && f->ny0 > 0 && f->max_level >= 0 && f->max_level <= 20 &&
           f->hx0 > 0 && f->hy0 > 0 && std::isfinite(f->x0) && std::isfinite(f->y0) &&
           f->h_min >= 0 && ((int64_t)f->nx0 << f->max_level) < (1 << 29) &&
           ((int64_t)f->ny0 << f->max_level) < (1 << 29);
}

} // namespace swdg

using namespace swdg;

extern "C" {

int swdg_forest_flags(const swdg_forest* f, int64_t n, const int32_t* lij, const double* eta,
                      double theta_r, double theta_c, int8_t* flags) {
    if (!forest_valid(f) || n < 1 || !lij || !eta || !flags) return SWDG_EINVAL;
    Forest F{*f};
    std::vector<Leaf> L(n);
    for (int64_t k = 0; k < n; ++k) L[k] = Leaf{lij[3 * k], lij[3 * k + 1], lij[3 * k + 2]};
    F.flags(L, eta, theta_r, theta_c, flags);
    return SWDG_OK;
}

int swdg_forest_adapt(const swdg_forest* f, int64_t n, const int32_t* lij, const int8_t* flags,
                      int64_t cap, int32_t* lij_out, int64_t* n_out) {
    if (!forest_valid(f) || n < 1 || !lij || !flags || !n_out) return SWDG_EINVAL;
    Forest F{*f};
    std::vector<Leaf> L(n);
    for (int64_t k = 0; k < n; ++k) {
        L[k] = Leaf{lij[3 * k], lij[3 * k + 1], lij[3 * k + 2]};
        if (L[k].l < 0 || L[k].l > f->max_level) return SWDG_EINVAL;
    }
    std::vector<Leaf> out = F.adapt(L, flags);
    *n_out = (int64_t)out.size();
    if ((int64_t)out.size() > cap || !lij_out) return SWDG_EINVAL;
    for (size_t k = 0; k < out.size(); ++k) {
        lij_out[3 * k] = out[k].l;
        lij_out[3 * k + 1] = out[k].i;
        lij_out[3 * k + 2] = out[k].j;
    }
    return SWDG_OK;
}

int swdg_forest_mesh(const swdg_forest* f, int64_t n, const int32_t* lij, double* x0y0,
                     double* hxhy, int32_t* nbr) {
    if (!forest_valid(f) || n < 1 || !lij || !x0y0 || !hxhy || !nbr) return SWDG_EINVAL;
    Forest F{*f};
    std::vector<Leaf> L(n);
    for (int64_t k = 0; k < n; ++k) L[k] = Leaf{lij[3 * k], lij[3 * k + 1], lij[3 * k + 2]};
    try {
        F.mesh(L, x0y0, hxhy, nbr);
    } catch (...) { // a leaf set that is not 2:1 balanced has a face without its leaves
        return SWDG_EINVAL;
    }
    return SWDG_OK;
}

} // extern "C"
