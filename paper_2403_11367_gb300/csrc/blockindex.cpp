// blockindex.cpp -- see blockindex.h.
#include "blockindex.h"

#include <algorithm>
#include <cmath>
#include <numeric>

namespace reloc {

void BlockIndex::build(const float *means, int64_t n, double B_, std::vector<int64_t> &order)
{
    B = B_;
    std::vector<int64_t> kx(n), ky(n);
    for (int64_t i = 0; i < n; ++i) {
        kx[i] = (int64_t)std::floor((double)means[3 * i] / B);
        ky[i] = (int64_t)std::floor((double)means[3 * i + 1] / B);
    }
    order.resize(n);
    std::iota(order.begin(), order.end(), (int64_t)0);
    std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
        return kx[a] != kx[b] ? kx[a] < kx[b] : ky[a] < ky[b];
    });
    bx.clear(); by.clear(); begin.clear(); end.clear(); cx.clear(); cy.clear();
    for (int64_t p = 0; p < n;) {
        int64_t q = p;
        const int64_t X = kx[order[p]], Y = ky[order[p]];
        while (q < n && kx[order[q]] == X && ky[order[q]] == Y) ++q;
        bx.push_back(X); by.push_back(Y); begin.push_back(p); end.push_back(q);
        cx.push_back((X + 0.5) * B); cy.push_back((Y + 0.5) * B);
        p = q;
    }
    // implicit balanced KD-tree: the median of each range is its node
    kd.resize(bx.size());
    std::iota(kd.begin(), kd.end(), 0);
    struct Builder {
        BlockIndex *self;
        void operator()(int lo, int hi, int axis) {
            if (hi - lo <= 1) return;
            int mid = (lo + hi) / 2;
            const std::vector<double> &c = axis ? self->cy : self->cx;
            std::nth_element(self->kd.begin() + lo, self->kd.begin() + mid, self->kd.begin() + hi,
                             [&](int a, int b) { return c[a] < c[b]; });
            (*this)(lo, mid, axis ^ 1);
            (*this)(mid + 1, hi, axis ^ 1);
        }
    } builder{this};
    builder(0, (int)kd.size(), 0);
}

void BlockIndex::range(double x, double y, double r, std::vector<int> &out) const
{
    out.clear();
    struct Walker {
        const BlockIndex *s;
        double x, y, r;
        std::vector<int> *out;
        void operator()(int lo, int hi, int axis) {
            if (lo >= hi) return;
            int mid = (lo + hi) / 2;
            int b = s->kd[mid];
            double dx = s->cx[b] - x, dy = s->cy[b] - y;
            if (std::sqrt(dx * dx + dy * dy) <= r) out->push_back(b);
            double diff = axis ? y - s->cy[b] : x - s->cx[b];
            // left subtree holds coordinates <= the node's, right >= it
            if (diff <= r) (*this)(lo, mid, axis ^ 1);
            if (-diff <= r) (*this)(mid + 1, hi, axis ^ 1);
        }
    } walker{this, x, y, r, &out};
    walker(0, (int)kd.size(), 0);
    std::sort(out.begin(), out.end());
}

}  // namespace reloc
