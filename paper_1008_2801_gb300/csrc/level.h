// level.h -- geometry of a coupled level (host code): ghost-exchange records
// from box intersections.
#pragma once

#include <array>
#include <vector>

#include "common.cuh"

namespace mg {

int set_error(int code, const char *fmt, ...);

// A box of a level: cells lo[d] .. lo[d] + n[d] - 1 in level coordinates.
struct Brick {
    int lo[3];
    int n[3];
};

// 1 and the first overlapping pair (*a < *b) if two boxes share a cell, else 0.
int level_check_disjoint(const std::vector<Brick> &B, int *a, int *b);

// Every patch where a box's guard layer (the cells just outside one of its
// six faces; no edges or corners) meets another box: dst = the box whose
// guard cells are filled, src = the box that owns those cells.  Ordered by
// dst, face, src.  brute: test all pairs instead of the region bins.
std::vector<ExchRec> level_exchange(const std::vector<Brick> &B, bool brute = false);

// Patches of a single box whose axes d with period[d] > 0 are periodic with
// that period: the guard layer of a periodic face is filled from the box's
// own cells at the opposite face (src = dst = 0).
std::vector<ExchRec> periodic_exchange(const Brick &b, const int period[3]);

}  // namespace mg
