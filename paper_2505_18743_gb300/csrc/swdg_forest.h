// swdg_forest.h -- host-side quadtree forest of dynamic h-adaptation (see
// swdg_forest.cu), shared by the C-ABI's forest functions and the context's
// adaptation step.
#pragma once
#include <cstdint>
#include <vector>

#include "../../include/swdg.h"

namespace swdg {

struct Leaf {
    int32_t l, i, j; // level, column and row on the grid of that level
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
