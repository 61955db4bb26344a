// The H5MD layout of a handle's state (H5MD 1.1: the /h5md metadata group,
// time-dependent particle elements of one frame with step, time and value,
// the box with its boundary and edges, connectivity), and the random-number
// checkpoint: the Philox noise is a function of (seed, particle id, step), so
// the replicas' seeds and the step number restore it.  Paper "New features":
// H5MD output and the checkpoint of the random number generator.
//
//   /h5md                 version = {1, 1}; author (name), creator (name, version)
//   /particles/<g>/box    dimension = 3, boundary = periodic x 3; edges [3]
//   /particles/<g>/position, velocity, image   step [1], time [1], value [1][n][3]
//   /particles/<g>/force  the same, when the handle holds the step's total force
//   /particles/<g>/species                     [n] particle types
//   /connectivity/<g>/bonds                    [n_bonds][2] local ids
//   /parameters/espp      step, time, precision, lees_edwards, shear_rate; seeds [R]
// with <g> = "all" for a single system, "replica_<r>" for a batch.
#include <algorithm>
#include <cstring>

#include "h5md.h"

namespace espp {
namespace {
using h5::Attr;
using h5::Node;
using h5::Type;

template <class V>
std::vector<uint8_t> bytes_of(const V* p, size_t n) {
    std::vector<uint8_t> b(n * sizeof(V));
    if (n) memcpy(b.data(), p, b.size());
    return b;
}

Type t_f64() { return Type{Type::FLOAT, 8, true}; }
Type t_i32() { return Type{Type::INT, 4, true}; }
Type t_i64() { return Type{Type::INT, 8, true}; }
Type t_u64() { return Type{Type::INT, 8, false}; }

Node dataset(const std::string& name, Type t, std::vector<uint64_t> dims, std::vector<uint8_t> data,
             bool scalar = false) {
    Node n;
    n.name = name;
    n.is_group = false;
    n.type = t;
    n.dims = std::move(dims);
    n.scalar = scalar;
    n.data = std::move(data);
    return n;
}

Attr attr(const std::string& name, Type t, std::vector<uint64_t> dims, std::vector<uint8_t> data,
          bool scalar = false) {
    Attr a;
    a.name = name;
    a.type = t;
    a.dims = std::move(dims);
    a.scalar = scalar;
    a.data = std::move(data);
    return a;
}

Attr attr_str(const std::string& name, const std::vector<std::string>& v, bool scalar) {
    size_t len = 1;
    for (const std::string& s : v) len = std::max(len, s.size() + 1);
    std::vector<uint8_t> d(len * v.size(), 0);
    for (size_t k = 0; k < v.size(); ++k) memcpy(d.data() + k * len, v[k].data(), v[k].size());
    return attr(name, Type{Type::STRING, (uint32_t)len, false}, {(uint64_t)v.size()}, d, scalar);
}

// a time-dependent element of one frame
Node element(const std::string& name, int64_t step, double time, Node value) {
    Node g;
    g.name = name;
    g.is_group = true;
    g.children.push_back(dataset("step", t_i64(), {1}, bytes_of(&step, 1)));
    g.children.push_back(dataset("time", t_f64(), {1}, bytes_of(&time, 1)));
    value.name = "value";
    g.children.push_back(std::move(value));
    return g;
}

std::string group_name(size_t r, size_t R) { return R == 1 ? "all" : "replica_" + std::to_string(r); }

// a dataset of the given class, element size and shape whose data hold exactly
// that many elements (the element count formed without overflow: every
// partial product stays within the data's size)
bool shaped(const Node* n, Type::Cls cls, uint32_t size, const std::vector<uint64_t>& dims) {
    if (!n || n->is_group || n->type.cls != cls || n->type.size != size || n->dims != dims || size == 0)
        return false;
    const uint64_t cap = n->data.size() / size;
    uint64_t count = 1;
    for (uint64_t d : dims) {
        if (d != 0 && count > cap / d) return false;
        count *= d;
    }
    return n->data.size() == count * size;
}

const Attr* attr_of(const Node* n, const std::string& name) {
    if (!n) return nullptr;
    for (const Attr& a : n->attrs)
        if (a.name == name) return &a;
    return nullptr;
}

template <class V>
bool scalar_of(const Node* n, const std::string& name, V& out) {
    const Attr* a = attr_of(n, name);
    if (!a || a->data.size() != sizeof(V)) return false;
    memcpy(&out, a->data.data(), sizeof(V));
    return true;
}
}  // namespace

int h5md_write(const char* path, const H5mdState& st, std::string& err) {
    Node root;
    root.is_group = true;
    {
        Node& h = root.group("h5md");
        const int32_t version[2] = {1, 1};
        h.attrs.push_back(attr("version", t_i32(), {2}, bytes_of(version, 2)));
        h.group("author").attrs.push_back(attr_str("name", {"espp GB300 library"}, true));
        Node& c = h.group("creator");
        c.attrs.push_back(attr_str("name", {"paper_2608_14911_gb300"}, true));
        c.attrs.push_back(attr_str("version", {"2"}, true));
    }
    {
        Node& parts = root.group("particles");
        for (size_t r = 0; r < st.reps.size(); ++r) {
            const H5mdReplica& rp = st.reps[r];
            const uint64_t n = (uint64_t)rp.n;
            Node g;
            g.name = group_name(r, st.reps.size());
            g.is_group = true;
            Node box;
            box.name = "box";
            box.is_group = true;
            const int32_t dim = 3;
            box.attrs.push_back(attr("dimension", t_i32(), {}, bytes_of(&dim, 1), true));
            box.attrs.push_back(attr_str("boundary", {"periodic", "periodic", "periodic"}, false));
            box.children.push_back(dataset("edges", t_f64(), {3}, bytes_of(rp.box, 3)));
            g.children.push_back(std::move(box));
            g.children.push_back(
                element("position", st.step, st.time, dataset("value", t_f64(), {1, n, 3}, bytes_of(rp.x.data(), 3 * n))));
            g.children.push_back(
                element("velocity", st.step, st.time, dataset("value", t_f64(), {1, n, 3}, bytes_of(rp.v.data(), 3 * n))));
            g.children.push_back(
                element("image", st.step, st.time, dataset("value", t_i32(), {1, n, 3}, bytes_of(rp.img.data(), 3 * n))));
            if (!rp.f.empty())
                g.children.push_back(
                    element("force", st.step, st.time, dataset("value", t_f64(), {1, n, 3}, bytes_of(rp.f.data(), 3 * n))));
            g.children.push_back(dataset("species", t_i32(), {n}, bytes_of(rp.species.data(), n)));
            parts.children.push_back(std::move(g));
        }
    }
    {
        Node& con = root.group("connectivity");
        for (size_t r = 0; r < st.reps.size(); ++r) {
            const H5mdReplica& rp = st.reps[r];
            Node g;
            g.name = group_name(r, st.reps.size());
            g.is_group = true;
            g.children.push_back(dataset("bonds", t_i64(), {(uint64_t)rp.bonds.size() / 2, 2},
                                         bytes_of(rp.bonds.data(), rp.bonds.size())));
            con.children.push_back(std::move(g));
        }
    }
    {
        Node& par = root.group("parameters");
        Node e;
        e.name = "espp";
        e.is_group = true;
        e.attrs.push_back(attr("step", t_i64(), {}, bytes_of(&st.step, 1), true));
        e.attrs.push_back(attr("time", t_f64(), {}, bytes_of(&st.time, 1), true));
        e.attrs.push_back(attr("precision", t_i32(), {}, bytes_of(&st.precision, 1), true));
        e.attrs.push_back(attr("lees_edwards", t_i32(), {}, bytes_of(&st.lees_edwards, 1), true));
        e.attrs.push_back(attr("shear_rate", t_f64(), {}, bytes_of(&st.shear_rate, 1), true));
        std::vector<uint64_t> seeds;
        for (const H5mdReplica& rp : st.reps) seeds.push_back(rp.seed);
        e.children.push_back(dataset("seeds", t_u64(), {(uint64_t)seeds.size()}, bytes_of(seeds.data(), seeds.size())));
        par.children.push_back(std::move(e));
    }
    return h5::write_file(path, root, err);
}

int h5md_read(const char* path, H5mdState& st, std::string& err) {
    Node root;
    if (h5::read_file(path, root, err)) return -1;
    const Node* h = root.find("h5md");
    const Attr* ver = attr_of(h, "version");
    int32_t v[2] = {0, 0};
    if (!ver || ver->data.size() != 8) {
        err = "no /h5md version: not an H5MD file";
        return -1;
    }
    memcpy(v, ver->data.data(), 8);
    if (v[0] != 1) {
        err = "unsupported H5MD major version";
        return -1;
    }
    const Node* e = root.find("parameters/espp");
    if (!e || !scalar_of(e, "step", st.step) || !scalar_of(e, "time", st.time) ||
        !scalar_of(e, "precision", st.precision) || !scalar_of(e, "lees_edwards", st.lees_edwards) ||
        !scalar_of(e, "shear_rate", st.shear_rate)) {
        err = "missing /parameters/espp";
        return -1;
    }
    const Node* seeds = e->find("seeds");
    if (!seeds || seeds->dims.size() != 1 || !shaped(seeds, Type::INT, 8, {seeds->dims[0]}) ||
        seeds->dims[0] == 0) {
        err = "missing replica seeds";
        return -1;
    }
    const size_t R = (size_t)seeds->dims[0];
    st.reps.assign(R, H5mdReplica());
    for (size_t r = 0; r < R; ++r) {
        H5mdReplica& rp = st.reps[r];
        memcpy(&rp.seed, seeds->data.data() + 8 * r, 8);
        const std::string g = "particles/" + group_name(r, R);
        const Node* edges = root.find(g + "/box/edges");
        const Node* sp = root.find(g + "/species");
        if (!shaped(edges, Type::FLOAT, 8, {3}) || !sp || sp->is_group || sp->dims.size() != 1) {
            err = "missing box or species of " + g;
            return -1;
        }
        memcpy(rp.box, edges->data.data(), 24);
        rp.n = (int64_t)sp->dims[0];
        const uint64_t n = (uint64_t)rp.n;
        const Node* x = root.find(g + "/position/value");
        const Node* vel = root.find(g + "/velocity/value");
        const Node* img = root.find(g + "/image/value");
        if (!shaped(x, Type::FLOAT, 8, {1, n, 3}) || !shaped(vel, Type::FLOAT, 8, {1, n, 3}) ||
            !shaped(img, Type::INT, 4, {1, n, 3}) || !shaped(sp, Type::INT, 4, {n})) {
            err = "particle elements of " + g + " missing or of the wrong shape";
            return -1;
        }
        rp.x.resize(3 * n);
        rp.v.resize(3 * n);
        rp.img.resize(3 * n);
        rp.species.resize(n);
        memcpy(rp.x.data(), x->data.data(), x->data.size());
        memcpy(rp.v.data(), vel->data.data(), vel->data.size());
        memcpy(rp.img.data(), img->data.data(), img->data.size());
        memcpy(rp.species.data(), sp->data.data(), sp->data.size());
        if (const Node* f = root.find(g + "/force/value")) {
            if (!shaped(f, Type::FLOAT, 8, {1, n, 3})) {
                err = "force element of " + g + " of the wrong shape";
                return -1;
            }
            rp.f.resize(3 * n);
            memcpy(rp.f.data(), f->data.data(), f->data.size());
        }
        const Node* bonds = root.find("connectivity/" + group_name(r, R) + "/bonds");
        if (bonds && bonds->dims.size() == 2 && shaped(bonds, Type::INT, 8, {bonds->dims[0], 2})) {
            rp.bonds.resize(2 * (size_t)bonds->dims[0]);
            if (!rp.bonds.empty()) memcpy(rp.bonds.data(), bonds->data.data(), bonds->data.size());
        }
    }
    return 0;
}

}  // namespace espp
