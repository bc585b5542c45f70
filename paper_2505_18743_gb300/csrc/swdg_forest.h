// swdg_forest.h -- host-side quadtree forest of dynamic h-adaptation (see
// swdg_forest.cu), shared by the C-ABI's forest functions and the context's
// adaptation step.
#pragma once
#include <cstdint>
#include <unordered_map>
#include <vector>

#include "../../include/swdg.h"

namespace swdg {

struct Leaf {
    int32_t l, i, j; // level, column and row on the grid of that level
};

// index of the leaf that is cell (l, i, j), -1 if none: one int32 per cell
// of every level while they fit in 256 MB, else a hash map
class CellIndex {
  public:
    explicit CellIndex(const swdg_forest& f);
    void set(int l, int64_t i, int64_t j, int32_t v);
    int32_t get(int l, int64_t i, int64_t j) const;

  private:
    bool dense_ = false;
    std::vector<std::vector<int32_t>> grid_;
    std::vector<int64_t> nx_;
    std::unordered_map<uint64_t, int32_t> hash_;
};

struct Forest {
    swdg_forest f;
    bool wrap(int l, int64_t i, int64_t j, int64_t& ii, int64_t& jj) const;
    void flags(const std::vector<Leaf>& leaves, const double* eta, double theta_r, double theta_c,
               int8_t* out) const;
    std::vector<Leaf> adapt(const std::vector<Leaf>& leaves, const int8_t* flags) const;
    uint64_t morton(const Leaf& c) const;
    void order(std::vector<Leaf>& leaves) const;
    void mesh(const std::vector<Leaf>& leaves, double* x0y0, double* hxhy, int32_t* nbr) const;
    bool leaves_of(int64_t n, const double* x0y0, const double* hxhy, std::vector<Leaf>& out) const;
};

bool forest_valid(const swdg_forest* f);

} // namespace swdg
