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

// a set of cells of the forest: one occupancy byte per cell of every level
// while the levels fit in 256 MB (the usual case), else a hash set
class CellSet {
  public:
    explicit CellSet(const swdg_forest& f) {
        int64_t tot = 0;
        for (int l = 0; l <= f.max_level; ++l) tot += ((int64_t)f.nx0 << l) * ((int64_t)f.ny0 << l);
        dense_ = tot <= (int64_t)1 << 28;
        if (dense_) {
            grid_.resize(f.max_level + 1);
            nx_.resize(f.max_level + 1);
            for (int l = 0; l <= f.max_level; ++l) {
                nx_[l] = (int64_t)f.nx0 << l;
                grid_[l].assign((size_t)nx_[l] * ((int64_t)f.ny0 << l), 0);
            }
        }
    }
    bool count(uint64_t key) const {
        if (!dense_) return hash_.count(key) != 0;
        const int l = (int)(key >> 58);
        if (l < 0 || l >= (int)grid_.size()) return false;
        const int64_t i = (int64_t)((key >> 29) & ((1ull << 29) - 1)), j = (int64_t)(key & ((1ull << 29) - 1));
        return grid_[l][(size_t)(i + nx_[l] * j)] != 0;
    }
    void insert(uint64_t key) {
        if (!dense_) {
            hash_.insert(key);
            return;
        }
        const int l = (int)(key >> 58);
        const int64_t i = (int64_t)((key >> 29) & ((1ull << 29) - 1)), j = (int64_t)(key & ((1ull << 29) - 1));
        grid_[l][(size_t)(i + nx_[l] * j)] = 1;
    }
    void erase(uint64_t key) {
        if (!dense_) {
            hash_.erase(key);
            return;
        }
        const int l = (int)(key >> 58);
        const int64_t i = (int64_t)((key >> 29) & ((1ull << 29) - 1)), j = (int64_t)(key & ((1ull << 29) - 1));
        grid_[l][(size_t)(i + nx_[l] * j)] = 0;
    }

  private:
    bool dense_ = false;
    std::vector<std::vector<uint8_t>> grid_;
    std::vector<int64_t> nx_;
    std::unordered_set<uint64_t> hash_;
};

CellIndex::CellIndex(const swdg_forest& f) {
    int64_t tot = 0;
    for (int l = 0; l <= f.max_level; ++l) tot += ((int64_t)f.nx0 << l) * ((int64_t)f.ny0 << l);
    dense_ = tot <= (int64_t)1 << 26;
    if (dense_) {
        grid_.resize(f.max_level + 1);
        nx_.resize(f.max_level + 1);
        for (int l = 0; l <= f.max_level; ++l) {
            nx_[l] = (int64_t)f.nx0 << l;
            grid_[l].assign((size_t)nx_[l] * ((int64_t)f.ny0 << l), -1);
        }
    }
}

void CellIndex::set(int l, int64_t i, int64_t j, int32_t v) {
    if (dense_) grid_[l][(size_t)(i + nx_[l] * j)] = v;
    else hash_[pack(l, i, j)] = v;
}

int32_t CellIndex::get(int l, int64_t i, int64_t j) const {
    if (l < 0) return -1;
    if (dense_) {
        if (l >= (int)grid_.size()) return -1;
        return grid_[l][(size_t)(i + nx_[l] * j)];
    }
    auto it = hash_.find(pack(l, i, j));
    return it == hash_.end() ? -1 : it->second;
}

// the leaf covering cell (l, i, j) if it is that cell or an ancestor
static bool covering(const CellSet& S, int l, int64_t i, int64_t j, Leaf* out) {
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
    CellSet S(f), marked(f);
    std::vector<uint64_t> live; // every key ever inserted into S (removed ones are skipped)
    live.reserve(leaves.size() * 2);
    auto add = [&](uint64_t key) {
        S.insert(key);
        live.push_back(key);
    };
    for (size_t k = 0; k < leaves.size(); ++k) {
        const Leaf c = leaves[k];
        if (fl[k] == 1) {
            for (int b = 0; b < 2; ++b)
                for (int a = 0; a < 2; ++a) add(pack(c.l + 1, 2 * c.i + a, 2 * c.j + b));
        } else {
            add(pack(c.l, c.i, c.j));
        }
        if (fl[k] == -1) marked.insert(pack(c.l, c.i, c.j));
    }
    // four siblings, all leaves and all marked, merge into their parent
    CellSet done(f);
    for (size_t k = 0; k < leaves.size(); ++k) {
        if (fl[k] != -1) continue;
        const Leaf c = leaves[k];
        const int l = c.l - 1;
        const int64_t pi = c.i >> 1, pj = c.j >> 1;
        const uint64_t pk = pack(l, pi, pj);
        if (done.count(pk)) continue;
        done.insert(pk);
        bool all = true;
        for (int b = 0; b < 2 && all; ++b)
            for (int a = 0; a < 2 && all; ++a) {
                const uint64_t ck = pack(l + 1, 2 * pi + a, 2 * pj + b);
                all = S.count(ck) && marked.count(ck);
            }
        if (!all) continue;
        for (int b = 0; b < 2; ++b)
            for (int a = 0; a < 2; ++a) S.erase(pack(l + 1, 2 * pi + a, 2 * pj + b));
        add(pk);
    }
    // 2:1 balance: split every leaf whose face neighbour region holds leaves
    // two or more levels finer, until none does
    bool changed = true;
    while (changed) {
        changed = false;
        const size_t nlive = live.size();
        for (size_t q = 0; q < nlive; ++q) {
            const uint64_t key = live[q];
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
                    for (int a = 0; a < 2; ++a) add(pack(l + 1, 2 * i + a, 2 * j + b));
                changed = true;
                break;
            }
        }
    }
    std::vector<Leaf> out;
    CellSet seen(f);
    for (uint64_t key : live) {
        if (!S.count(key) || seen.count(key)) continue;
        seen.insert(key);
        out.push_back(Leaf{(int)(key >> 58), (int32_t)((key >> 29) & ((1ull << 29) - 1)),
                           (int32_t)(key & ((1ull << 29) - 1))});
    }
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
    std::vector<std::pair<uint64_t, Leaf>> kl(leaves.size());
    for (size_t k = 0; k < leaves.size(); ++k) kl[k] = {morton(leaves[k]), leaves[k]};
    std::sort(kl.begin(), kl.end(),
              [](const std::pair<uint64_t, Leaf>& a, const std::pair<uint64_t, Leaf>& b) {
                  return a.first < b.first;
              });
    for (size_t k = 0; k < leaves.size(); ++k) leaves[k] = kl[k].second;
}

void Forest::mesh(const std::vector<Leaf>& leaves, double* x0y0, double* hxhy, int32_t* nbr) const {
    CellIndex index(f);
    for (size_t k = 0; k < leaves.size(); ++k)
        index.set(leaves[k].l, leaves[k].i, leaves[k].j, (int32_t)k);
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
            int32_t v = index.get(c.l, ii, jj);
            if (v >= 0) {
                s[0] = v;
                continue;
            }
            v = index.get(c.l - 1, ii >> 1, jj >> 1);
            if (v >= 0) {
                s[0] = v;
                continue;
            }
            if (c.l + 1 > f.max_level) throw 1; // no finer leaves can exist: not balanced
            int32_t v0, v1;
            if (DIR[d][0] != 0) {
                const int a = DIR[d][0] > 0 ? 0 : 1;
                v0 = index.get(c.l + 1, 2 * ii + a, 2 * jj);
                v1 = index.get(c.l + 1, 2 * ii + a, 2 * jj + 1);
            } else {
                const int b = DIR[d][1] > 0 ? 0 : 1;
                v0 = index.get(c.l + 1, 2 * ii, 2 * jj + b);
                v1 = index.get(c.l + 1, 2 * ii + 1, 2 * jj + b);
            }
            if (v0 < 0 || v1 < 0) throw 1; // the face is not 2:1 balanced
            s[0] = v0;
            s[1] = v1;
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
