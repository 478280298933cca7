// octree.cpp -- GIGAQBX octree and interaction lists (Sec. 3.1-3.2), used to
// build the near-field pair lists that feed the TSQBX step.
//
// Input tooling: it produces geometry/list inputs shared by the CPU oracle and
// the GPU library, and holds none of the expansion arithmetic.
//
// Readings of the definitions (each is listed with its reason in the design
// notes):
//  * Two boxes are "adjacent" when their closed boxes intersect; this also
//    covers a box and its own descendants (they overlap), which keeps the
//    descendants of a target box out of its List 3.
//  * a < TCR(b) ("a adequately separated from the TCR of b"): the center of a
//    lies outside the ball TCR(b) and at l2 distance >= 3|a| from its surface.
//  * TCR(a) < b: the l-infinity distance from the center of a to the box b is
//    at least 3|a|(1+t_f) (the sufficient check the paper uses).
//  * Empty children are not created, so a leaf set need not tile the root.
//  * Box geometry is dyadic (power-of-two root width, grid-aligned center), so
//    adjacency and colleague tests are exact in double precision.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace {

struct Box {
    int level = 0;
    double c[3] = {0, 0, 0};
    double h = 0;                 // l-infinity radius (half width)
    int parent = -1;
    int child[8] = {-1, -1, -1, -1, -1, -1, -1, -1};
    bool leaf = true;
    int src_begin = 0, src_end = 0;   // sources of the whole subtree (sorted order)
    std::vector<int> own_src;     // during build (leaf sources)
    std::vector<int> own_ctr;     // owned QBX centers
    bool target = false;          // owns a center
    bool target_or_anc = false;   // target box or ancestor of one
};

struct Tree {
    std::vector<Box> boxes;
    std::vector<int> src_perm;    // sorted position -> original index
    std::vector<int> ctr_box;     // original center -> owning box
    double t_f = 0.9;
    int n_mpole = 0;
    // lists, kind -> per box vector of boxes
    std::vector<std::vector<int>> lists[8];
    std::vector<std::vector<int>> near_b, near_e;   // merged source ranges per box
};

enum { L1 = 0, L3CLOSE = 1, L3FAR = 2, L4CLOSE = 3, L2 = 4, L4FAR = 5, L3RAW = 6, L4RAW = 7 };

bool adjacent(const Box &a, const Box &b)
{
    for (int k = 0; k < 3; ++k)
        if (std::fabs(a.c[k] - b.c[k]) > a.h + b.h) return false;
    return true;
}

// same-level box d is a 2-colleague of b (inside the 2-near neighborhood)
bool colleague2(const Box &d, const Box &b)
{
    for (int k = 0; k < 3; ++k)
        if (std::fabs(d.c[k] - b.c[k]) > 4.0 * b.h) return false;
    return true;
}

double tcr_radius(const Tree &T, const Box &b) { return std::sqrt(3.0) * b.h * (1.0 + T.t_f); }

// a < TCR(b)
bool sep_box_tcr(const Tree &T, const Box &a, const Box &b)
{
    double d2 = 0;
    for (int k = 0; k < 3; ++k) d2 += (a.c[k] - b.c[k]) * (a.c[k] - b.c[k]);
    return std::sqrt(d2) - tcr_radius(T, b) >= 3.0 * a.h;
}

// TCR(a) < b, by the l-infinity sufficient check
bool sep_tcr_box(const Tree &T, const Box &a, const Box &b)
{
    double dist = 0;
    for (int k = 0; k < 3; ++k) dist = std::max(dist, std::fabs(a.c[k] - b.c[k]) - b.h);
    return dist >= 3.0 * a.h * (1.0 + T.t_f);
}

int nsrc(const Box &b) { return b.src_end - b.src_begin; }

void build_tree(Tree &T, int64_t n_src, const double *sx, int64_t n_ctr, const double *cx,
                const double *cr, int n_max)
{
    // bounding cube of sources and QBX balls
    double lo[3], hi[3];
    for (int k = 0; k < 3; ++k) { lo[k] = 1e300; hi[k] = -1e300; }
    for (int64_t i = 0; i < n_src; ++i)
        for (int k = 0; k < 3; ++k) {
            lo[k] = std::min(lo[k], sx[k * n_src + i]);
            hi[k] = std::max(hi[k], sx[k * n_src + i]);
        }
    for (int64_t i = 0; i < n_ctr; ++i)
        for (int k = 0; k < 3; ++k) {
            lo[k] = std::min(lo[k], cx[k * n_ctr + i] - cr[i]);
            hi[k] = std::max(hi[k], cx[k * n_ctr + i] + cr[i]);
        }
    double half = 0;
    for (int k = 0; k < 3; ++k) half = std::max(half, 0.5 * (hi[k] - lo[k]));
    double H = std::ldexp(1.0, (int)std::ceil(std::log2(std::max(half, 1e-30))));
    double q = H / 1024.0;
    if (half + q > H) { H *= 2.0; q *= 2.0; }   // room for the grid-aligned center
    Box root;
    for (int k = 0; k < 3; ++k) root.c[k] = std::round(0.5 * (lo[k] + hi[k]) / q) * q;
    root.h = H;
    for (int64_t i = 0; i < n_src; ++i) root.own_src.push_back((int)i);
    for (int64_t i = 0; i < n_ctr; ++i) root.own_ctr.push_back((int)i);
    T.boxes.push_back(root);

    // breadth-first splitting
    for (size_t bi = 0; bi < T.boxes.size(); ++bi) {
        if ((int)(T.boxes[bi].own_src.size() + T.boxes[bi].own_ctr.size()) <= n_max) continue;
        Box b = T.boxes[bi];   // copy (vector may reallocate)
        std::vector<int> kid_src[8], kid_ctr[8], stay;
        auto octant = [&](const double *p) {
            int o = 0;
            for (int k = 0; k < 3; ++k) if (p[k] >= b.c[k]) o |= 1 << k;
            return o;
        };
        for (int s : b.own_src) {
            double p[3] = {sx[s], sx[n_src + s], sx[2 * n_src + s]};
            kid_src[octant(p)].push_back(s);
        }
        double hh = 0.5 * b.h;
        double rt = std::sqrt(3.0) * hh * (1.0 + T.t_f);
        for (int c : b.own_ctr) {
            double p[3] = {cx[c], cx[n_ctr + c], cx[2 * n_ctr + c]};
            int o = octant(p);
            double kc[3], d2 = 0;
            for (int k = 0; k < 3; ++k) {
                kc[k] = b.c[k] + ((o >> k) & 1 ? hh : -hh);
                d2 += (p[k] - kc[k]) * (p[k] - kc[k]);
            }
            if (std::sqrt(d2) + cr[c] <= rt) kid_ctr[o].push_back(c);
            else stay.push_back(c);
        }
        bool any = false;
        for (int o = 0; o < 8; ++o) if (!kid_src[o].empty() || !kid_ctr[o].empty()) any = true;
        if (!any) continue;   // nothing can move down: stays a leaf
        T.boxes[bi].own_src.clear();
        T.boxes[bi].own_ctr = stay;
        T.boxes[bi].leaf = false;
        for (int o = 0; o < 8; ++o) {
            if (kid_src[o].empty() && kid_ctr[o].empty()) continue;
            Box k;
            k.level = b.level + 1;
            k.h = hh;
            for (int a = 0; a < 3; ++a) k.c[a] = b.c[a] + ((o >> a) & 1 ? hh : -hh);
            k.parent = (int)bi;
            k.own_src = std::move(kid_src[o]);
            k.own_ctr = std::move(kid_ctr[o]);
            T.boxes[bi].child[o] = (int)T.boxes.size();
            T.boxes.push_back(std::move(k));
        }
    }
    // depth-first source order
    T.src_perm.clear();
    // iterative DFS assigning each box the source range of its subtree
    struct Frame { int b; int next; };
    std::vector<Frame> st{{0, 0}};
    T.boxes[0].src_begin = 0;
    while (!st.empty()) {
        Frame &f = st.back();
        Box &b = T.boxes[f.b];
        if (f.next == 0) {
            b.src_begin = (int)T.src_perm.size();
            for (int s : b.own_src) T.src_perm.push_back(s);
        }
        bool pushed = false;
        while (f.next < 8) {
            int c = b.child[f.next++];
            if (c >= 0) { st.push_back({c, 0}); pushed = true; break; }
        }
        if (!pushed) {
            T.boxes[st.back().b].src_end = (int)T.src_perm.size();
            st.pop_back();
        }
    }
    T.ctr_box.assign((size_t)n_ctr, -1);
    for (size_t bi = 0; bi < T.boxes.size(); ++bi) {
        for (int c : T.boxes[bi].own_ctr) T.ctr_box[c] = (int)bi;
        if (!T.boxes[bi].own_ctr.empty()) {
            T.boxes[bi].target = true;
            for (int a = (int)bi; a >= 0; a = T.boxes[a].parent) T.boxes[a].target_or_anc = true;
        }
    }
}

// collect leaves adjacent to b (List 1)
void collect_adjacent_leaves(const Tree &T, int node, const Box &b, std::vector<int> &out)
{
    const Box &x = T.boxes[node];
    if (!adjacent(x, b)) return;
    if (x.leaf) { if (nsrc(x) > 0) out.push_back(node); return; }
    for (int c : x.child) if (c >= 0) collect_adjacent_leaves(T, c, b, out);
}

// same-level boxes inside the 2-near neighborhood of b (its 2-colleagues, b included)
void collect_colleagues(const Tree &T, int node, const Box &b, std::vector<int> &out)
{
    const Box &x = T.boxes[node];
    for (int k = 0; k < 3; ++k)
        if (std::fabs(x.c[k] - b.c[k]) > x.h + 5.0 * b.h) return;
    if (x.level == b.level) { if (colleague2(x, b)) out.push_back(node); return; }
    for (int c : x.child) if (c >= 0) collect_colleagues(T, c, b, out);
}

void list3_walk(const Tree &T, int node, const Box &b, std::vector<int> &out)
{
    const Box &d = T.boxes[node];
    if (nsrc(d) == 0) return;
    if (!adjacent(d, b)) { out.push_back(node); return; }
    if (d.leaf) return;
    for (int c : d.child) if (c >= 0) list3_walk(T, c, b, out);
}

void list3_classify(const Tree &T, int node, const Box &b, std::vector<int> &close,
                    std::vector<int> &far)
{
    const Box &w = T.boxes[node];
    if (nsrc(w) == 0) return;
    if (sep_box_tcr(T, w, b)) {            // List 3 far candidate
        if (nsrc(w) >= T.n_mpole) far.push_back(node);
        else close.push_back(node);        // all leaves below w are List 3 close
        return;
    }
    if (w.leaf) { close.push_back(node); return; }
    for (int c : w.child) if (c >= 0) list3_classify(T, c, b, close, far);
}

// List 4 (i): source leaves coarser than w, adjacent to parent(w), not adjacent to w
void list4_coarse(const Tree &T, int node, const Box &w, const Box &pw, std::vector<int> &out)
{
    const Box &x = T.boxes[node];
    if (x.level >= w.level || !adjacent(x, pw)) return;
    if (x.leaf) { if (nsrc(x) > 0 && !adjacent(x, w)) out.push_back(node); return; }
    for (int c : x.child) if (c >= 0) list4_coarse(T, c, w, pw, out);
}

void build_lists(Tree &T)
{
    size_t nb = T.boxes.size();
    for (auto &l : T.lists) l.assign(nb, {});
    std::vector<std::vector<int>> coll(nb);
    // 2-colleagues of every target/ancestor box and of their parents
    for (size_t b = 0; b < nb; ++b)
        if (T.boxes[b].target_or_anc) collect_colleagues(T, 0, T.boxes[b], coll[b]);
    // List 2 and raw List 4 for target-or-ancestor boxes (top-down order:
    // boxes are stored breadth first, so parents precede children)
    for (size_t b = 0; b < nb; ++b) {
        const Box &w = T.boxes[b];
        if (!w.target_or_anc) continue;
        if (w.parent >= 0) {
            const Box &pw = T.boxes[w.parent];
            for (int pc : coll[w.parent])
                for (int c : T.boxes[pc].child)
                    if (c >= 0 && !colleague2(T.boxes[c], w) && nsrc(T.boxes[c]) > 0)
                        T.lists[L2][b].push_back(c);
            list4_coarse(T, 0, w, pw, T.lists[L4RAW][b]);
        }
        for (int d : coll[b]) {
            const Box &x = T.boxes[d];
            if (x.leaf && nsrc(x) > 0 && !adjacent(x, w)) T.lists[L4RAW][b].push_back(d);
        }
        // List 4 close / far
        for (int a = (int)b; a >= 0; a = T.boxes[a].parent)
            for (int d : T.lists[L4RAW][a])
                if (!sep_tcr_box(T, w, T.boxes[d])) T.lists[L4CLOSE][b].push_back(d);
        for (int d : T.lists[L4RAW][b])
            if (sep_tcr_box(T, w, T.boxes[d])) T.lists[L4FAR][b].push_back(d);
        if (w.parent >= 0)
            for (int d : T.lists[L4CLOSE][w.parent])
                if (sep_tcr_box(T, w, T.boxes[d])) T.lists[L4FAR][b].push_back(d);
    }
    // Lists 1 and 3 for target boxes
    for (size_t b = 0; b < nb; ++b) {
        const Box &w = T.boxes[b];
        if (!w.target) continue;
        collect_adjacent_leaves(T, 0, w, T.lists[L1][b]);
        for (int cb : coll[b])
            for (int c : T.boxes[cb].child)
                if (c >= 0) list3_walk(T, c, w, T.lists[L3RAW][b]);
        for (int d : T.lists[L3RAW][b])
            list3_classify(T, d, w, T.lists[L3CLOSE][b], T.lists[L3FAR][b]);
    }
    // merged near-field source ranges: List 1 + List 3 close + List 4 close
    T.near_b.assign(nb, {});
    T.near_e.assign(nb, {});
    for (size_t b = 0; b < nb; ++b) {
        if (!T.boxes[b].target) continue;
        std::vector<std::pair<int, int>> r;
        for (int kind : {L1, L3CLOSE, L4CLOSE})
            for (int d : T.lists[kind][b]) r.push_back({T.boxes[d].src_begin, T.boxes[d].src_end});
        std::sort(r.begin(), r.end());
        for (auto &x : r) {
            if (x.first == x.second) continue;
            if (!T.near_b[b].empty() && T.near_e[b].back() == x.first) T.near_e[b].back() = x.second;
            else { T.near_b[b].push_back(x.first); T.near_e[b].push_back(x.second); }
        }
    }
}

}  // namespace

extern "C" {

void *oct_build(int64_t n_src, const double *src_xyz, int64_t n_ctr, const double *ctr_xyz,
                const double *ctr_radius, int n_max, double t_f, int n_mpole)
{
    if (n_src < 0 || n_ctr < 0 || n_max < 1 || t_f < 0) return nullptr;
    Tree *T = new Tree;
    T->t_f = t_f;
    T->n_mpole = n_mpole;
    build_tree(*T, n_src, src_xyz, n_ctr, ctr_xyz, ctr_radius, n_max);
    build_lists(*T);
    return T;
}

void oct_free(void *h) { delete static_cast<Tree *>(h); }

int64_t oct_n_boxes(void *h) { return (int64_t) static_cast<Tree *>(h)->boxes.size(); }

void oct_box_info(void *h, int32_t *level, double *center, double *halfwidth, int32_t *parent,
                  int32_t *src_begin, int32_t *src_end, int32_t *n_owned_ctr, int32_t *is_leaf)
{
    Tree &T = *static_cast<Tree *>(h);
    size_t nb = T.boxes.size();
    for (size_t b = 0; b < nb; ++b) {
        const Box &x = T.boxes[b];
        level[b] = x.level;
        for (int k = 0; k < 3; ++k) center[k * nb + b] = x.c[k];
        halfwidth[b] = x.h;
        parent[b] = x.parent;
        src_begin[b] = x.src_begin;
        src_end[b] = x.src_end;
        n_owned_ctr[b] = (int32_t)x.own_ctr.size();
        is_leaf[b] = x.leaf ? 1 : 0;
    }
}

void oct_src_perm(void *h, int32_t *perm)
{
    Tree &T = *static_cast<Tree *>(h);
    std::memcpy(perm, T.src_perm.data(), T.src_perm.size() * sizeof(int32_t));
}

void oct_ctr_box(void *h, int32_t *box)
{
    Tree &T = *static_cast<Tree *>(h);
    std::memcpy(box, T.ctr_box.data(), T.ctr_box.size() * sizeof(int32_t));
}

int64_t oct_list_nnz(void *h, int kind)
{
    Tree &T = *static_cast<Tree *>(h);
    if (kind < 0 || kind > 7) return -1;
    int64_t n = 0;
    for (auto &v : T.lists[kind]) n += (int64_t)v.size();
    return n;
}

int oct_list(void *h, int kind, int64_t *start, int32_t *boxes)
{
    Tree &T = *static_cast<Tree *>(h);
    if (kind < 0 || kind > 7) return -1;
    int64_t n = 0;
    start[0] = 0;
    for (size_t b = 0; b < T.boxes.size(); ++b) {
        for (int d : T.lists[kind][b]) boxes[n++] = d;
        start[b + 1] = n;
    }
    return 0;
}

int64_t oct_near_nnz(void *h)
{
    Tree &T = *static_cast<Tree *>(h);
    int64_t n = 0;
    for (auto &v : T.near_b) n += (int64_t)v.size();
    return n;
}

void oct_near_ranges(void *h, int64_t *start, int32_t *rb, int32_t *re)
{
    Tree &T = *static_cast<Tree *>(h);
    int64_t n = 0;
    start[0] = 0;
    for (size_t b = 0; b < T.boxes.size(); ++b) {
        for (size_t i = 0; i < T.near_b[b].size(); ++i) {
            rb[n] = T.near_b[b][i];
            re[n] = T.near_e[b][i];
            ++n;
        }
        start[b + 1] = n;
    }
}

}  // extern "C"
