// level.cu -- geometry of a coupled level: which cells of which box fill the
// guard cells of which other box (host code).
//
// A level is the union of disjoint boxes (paper Sec. 2: a MultiFAB holds data
// on the union of disjoint rectangular grids).  Filling a box's ghost cells
// needs the intersections of every box's ghost layer with the other boxes.
// Testing every pair costs O(N^2) for N boxes; the paper's hash sort bins the
// boxes into regions of index space at least as large as any box, keyed by
// the region that holds a box's lowest corner, so that a box can only touch
// boxes of its own or a neighbouring region: O(N + N^2/M) for M regions.  The
// records are computed once when a coupled solver is created and kept on the
// device with the solver's other launch data (the cached communication
// pattern).
#include <algorithm>
#include <cstdint>
#include <unordered_map>
#include <vector>

#include "level.h"

namespace mg {

static long long floor_div(long long a, long long b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

static long long bin_key(long long x, long long y, long long z)
{
    // 21 bits per coordinate (offset so that negative regions fit)
    const long long o = 1LL << 20;
    return ((x + o) << 42) | ((y + o) << 21) | (z + o);
}

// The guard layer of box b's face f (0..5 = x-, x+, y-, y+, z-, z+) as a
// half-open brick in level coordinates.
static void guard_slab(const Brick &b, int f, long long lo[3], long long hi[3])
{
    for (int d = 0; d < 3; ++d) {
        lo[d] = b.lo[d];
        hi[d] = (long long)b.lo[d] + b.n[d];
    }
    const int d = f / 2;
    if (f & 1) {
        lo[d] = hi[d];
        hi[d] = hi[d] + 1;
    } else {
        hi[d] = lo[d];
        lo[d] = lo[d] - 1;
    }
}

// Records for the slab of box b's face f intersected with box c.
static bool intersect(const Brick &b, int f, const Brick &c, ExchRec &r)
{
    long long lo[3], hi[3];
    guard_slab(b, f, lo, hi);
    long long ilo[3], ihi[3];
    for (int d = 0; d < 3; ++d) {
        ilo[d] = std::max(lo[d], (long long)c.lo[d]);
        ihi[d] = std::min(hi[d], (long long)c.lo[d] + c.n[d]);
        if (ilo[d] >= ihi[d]) return false;
    }
    r.di = (int)(ilo[0] - b.lo[0]);
    r.dj = (int)(ilo[1] - b.lo[1]);
    r.dk = (int)(ilo[2] - b.lo[2]);
    r.si = (int)(ilo[0] - c.lo[0]);
    r.sj = (int)(ilo[1] - c.lo[1]);
    r.sk = (int)(ilo[2] - c.lo[2]);
    r.ex = (int)(ihi[0] - ilo[0]);
    r.ey = (int)(ihi[1] - ilo[1]);
    r.ez = (int)(ihi[2] - ilo[2]);
    return true;
}

static bool overlap(const Brick &a, const Brick &b)
{
    for (int d = 0; d < 3; ++d)
        if (std::max(a.lo[d], b.lo[d]) >= std::min(a.lo[d] + a.n[d], b.lo[d] + b.n[d]))
            return false;
    return true;
}

// Candidate partners of every box: the boxes of its own region and the 26
// neighbouring ones.
static std::vector<std::vector<int>> candidates(const std::vector<Brick> &B)
{
    long long R[3] = {1, 1, 1};
    for (const Brick &b : B)
        for (int d = 0; d < 3; ++d) R[d] = std::max<long long>(R[d], b.n[d]);
    std::unordered_map<long long, std::vector<int>> bins;
    std::vector<std::array<long long, 3>> key(B.size());
    for (size_t i = 0; i < B.size(); ++i) {
        for (int d = 0; d < 3; ++d) key[i][d] = floor_div(B[i].lo[d], R[d]);
        bins[bin_key(key[i][0], key[i][1], key[i][2])].push_back((int)i);
    }
    std::vector<std::vector<int>> out(B.size());
    for (size_t i = 0; i < B.size(); ++i) {
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    auto it = bins.find(bin_key(key[i][0] + dx, key[i][1] + dy, key[i][2] + dz));
                    if (it == bins.end()) continue;
                    for (int c : it->second)
                        if (c != (int)i) out[i].push_back(c);
                }
        std::sort(out[i].begin(), out[i].end());
    }
    return out;
}

int level_check_disjoint(const std::vector<Brick> &B, int *a, int *b)
{
    const auto cand = candidates(B);
    for (size_t i = 0; i < B.size(); ++i)
        for (int c : cand[i])
            if (c > (int)i && overlap(B[i], B[c])) {
                *a = (int)i;
                *b = c;
                return 1;
            }
    return 0;
}

std::vector<ExchRec> level_exchange(const std::vector<Brick> &B, bool brute)
{
    std::vector<ExchRec> recs;
    std::vector<std::vector<int>> cand;
    if (!brute) cand = candidates(B);
    for (size_t i = 0; i < B.size(); ++i) {
        std::vector<int> all;
        if (brute) {
            for (size_t c = 0; c < B.size(); ++c)
                if (c != i) all.push_back((int)c);
        }
        const std::vector<int> &cs = brute ? all : cand[i];
        for (int f = 0; f < 6; ++f)
            for (int c : cs) {
                ExchRec r{};
                if (intersect(B[i], f, B[c], r)) {
                    r.dst = (int)i;
                    r.src = c;
                    recs.push_back(r);
                }
            }
    }
    return recs;
}

std::vector<ExchRec> periodic_exchange(const Brick &b, const int period[3])
{
    std::vector<ExchRec> recs;
    for (int f = 0; f < 6; ++f) {
        const int d = f / 2;
        if (period[d] <= 0) continue;
        Brick img = b;  // the box shifted by one period towards the face
        img.lo[d] += (f & 1) ? period[d] : -period[d];
        ExchRec r{};
        if (intersect(b, f, img, r)) {
            r.dst = 0;
            r.src = 0;
            // src coordinates are relative to the image: those are the box's own
            recs.push_back(r);
        }
    }
    return recs;
}

}  // namespace mg

extern "C" int mg_level_intersections(int nbox, const int (*lo)[3], const int (*n)[3],
                                      int brute, int *nrec, int *out, int cap)
{
    if (nbox < 0 || !nrec || (nbox > 0 && (!lo || !n)) || cap < 0 || (cap > 0 && !out))
        return mg::set_error(MG_ERR_INVALID_ARG, "bad argument");
    std::vector<mg::Brick> B(nbox);
    for (int b = 0; b < nbox; ++b)
        for (int d = 0; d < 3; ++d) {
            if (n[b][d] < 1)
                return mg::set_error(MG_ERR_INVALID_ARG, "box %d: dims must be >= 1", b);
            B[b].lo[d] = lo[b][d];
            B[b].n[d] = n[b][d];
        }
    int a = 0, c = 0;
    if (mg::level_check_disjoint(B, &a, &c))
        return mg::set_error(MG_ERR_INVALID_ARG, "boxes %d and %d overlap", a, c);
    const auto recs = mg::level_exchange(B, brute != 0);
    *nrec = (int)recs.size();
    for (int q = 0; q < std::min((int)recs.size(), cap); ++q) {
        const mg::ExchRec &r = recs[q];
        const int v[11] = {r.dst, r.src, r.di, r.dj, r.dk, r.si, r.sj, r.sk, r.ex, r.ey, r.ez};
        for (int e = 0; e < 11; ++e) out[11 * q + e] = v[e];
    }
    return MG_OK;
}
