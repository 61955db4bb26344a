// H5MD files (the HDF5-based molecular-data format the paper names among its
// new features, with the state and the random-number checkpoint) written and
// read without an HDF5 library.  This file holds a small HDF5 encoder and
// decoder for the subset H5MD needs here, built from the HDF5 file-format
// specification:
//   superblock version 2 (offsets and lengths of 8 bytes, a checksum);
//   object headers version 2 ("OHDR", one chunk, a checksum);
//   groups in compact form: a Link Info and a Group Info message, one Link
//     message per child (hard links);
//   datasets with contiguous storage: Dataspace (version 2), Datatype
//     (fixed-point, IEEE double, fixed-length ASCII string), Fill Value
//     (version 3) and Data Layout (version 3) messages;
//   attributes as Attribute messages (version 3) in the object header.
// Checksums are Bob Jenkins' lookup3 "hashlittle" with initial value 0, as
// the specification prescribes.  The decoder reads the files this encoder
// writes (it refuses anything else with a clear error); it is not a general
// HDF5 reader.
#include "h5md.h"

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <functional>

namespace espp {
namespace h5 {

static const uint64_t UNDEF = ~(uint64_t)0;

// ---- lookup3 hashlittle (Bob Jenkins, public domain algorithm) ---------------
static inline uint32_t rot(uint32_t x, int k) { return (x << k) | (x >> (32 - k)); }

uint32_t lookup3(const uint8_t* k, size_t length, uint32_t initval) {
    uint32_t a, b, c;
    a = b = c = 0xdeadbeefu + (uint32_t)length + initval;
    while (length > 12) {
        a += k[0] + ((uint32_t)k[1] << 8) + ((uint32_t)k[2] << 16) + ((uint32_t)k[3] << 24);
        b += k[4] + ((uint32_t)k[5] << 8) + ((uint32_t)k[6] << 16) + ((uint32_t)k[7] << 24);
        c += k[8] + ((uint32_t)k[9] << 8) + ((uint32_t)k[10] << 16) + ((uint32_t)k[11] << 24);
        // mix
        a -= c; a ^= rot(c, 4);  c += b;
        b -= a; b ^= rot(a, 6);  a += c;
        c -= b; c ^= rot(b, 8);  b += a;
        a -= c; a ^= rot(c, 16); c += b;
        b -= a; b ^= rot(a, 19); a += c;
        c -= b; c ^= rot(b, 4);  b += a;
        length -= 12;
        k += 12;
    }
    switch (length) {  // the last block: bytes added from the top down
        case 12: c += (uint32_t)k[11] << 24; [[fallthrough]];
        case 11: c += (uint32_t)k[10] << 16; [[fallthrough]];
        case 10: c += (uint32_t)k[9] << 8; [[fallthrough]];
        case 9: c += k[8]; [[fallthrough]];
        case 8: b += (uint32_t)k[7] << 24; [[fallthrough]];
        case 7: b += (uint32_t)k[6] << 16; [[fallthrough]];
        case 6: b += (uint32_t)k[5] << 8; [[fallthrough]];
        case 5: b += k[4]; [[fallthrough]];
        case 4: a += (uint32_t)k[3] << 24; [[fallthrough]];
        case 3: a += (uint32_t)k[2] << 16; [[fallthrough]];
        case 2: a += (uint32_t)k[1] << 8; [[fallthrough]];
        case 1: a += k[0]; break;
        case 0: return c;
    }
    // final
    c ^= b; c -= rot(b, 14);
    a ^= c; a -= rot(c, 11);
    b ^= a; b -= rot(a, 25);
    c ^= b; c -= rot(b, 16);
    a ^= c; a -= rot(c, 4);
    b ^= a; b -= rot(a, 14);
    c ^= b; c -= rot(b, 24);
    return c;
}

// ---- little-endian byte buffer --------------------------------------------------
struct Out {
    std::vector<uint8_t> b;
    void u8(uint32_t v) { b.push_back((uint8_t)v); }
    void u16(uint32_t v) { for (int i = 0; i < 2; ++i) b.push_back((uint8_t)(v >> (8 * i))); }
    void u32(uint32_t v) { for (int i = 0; i < 4; ++i) b.push_back((uint8_t)(v >> (8 * i))); }
    void u64(uint64_t v) { for (int i = 0; i < 8; ++i) b.push_back((uint8_t)(v >> (8 * i))); }
    void raw(const void* p, size_t n) {
        const uint8_t* q = static_cast<const uint8_t*>(p);
        b.insert(b.end(), q, q + n);
    }
};

// ---- datatype and dataspace messages ------------------------------------------------
static std::vector<uint8_t> type_msg(const Type& t) {
    Out o;
    if (t.cls == Type::INT) {
        o.u8(0x10);                    // version 1, class 0 (fixed-point)
        o.u8(t.is_signed ? 0x08 : 0);  // little-endian, signed bit
        o.u8(0);
        o.u8(0);
        o.u32(t.size);
        o.u16(0);             // bit offset
        o.u16(8 * t.size);    // bit precision
    } else if (t.cls == Type::FLOAT) {
        o.u8(0x11);           // version 1, class 1 (floating point)
        o.u8(0x20);           // little-endian, implied leading mantissa bit
        o.u8(63);             // sign bit position
        o.u8(0);
        o.u32(8);
        o.u16(0);             // bit offset
        o.u16(64);            // precision
        o.u8(52);             // exponent location
        o.u8(11);             // exponent size
        o.u8(0);              // mantissa location
        o.u8(52);             // mantissa size
        o.u32(1023);          // exponent bias
    } else {
        o.u8(0x13);           // version 1, class 3 (string)
        o.u8(0x00);           // null-terminated, ASCII
        o.u8(0);
        o.u8(0);
        o.u32(t.size);
    }
    return o.b;
}

static std::vector<uint8_t> space_msg(const std::vector<uint64_t>& dims, bool scalar) {
    Out o;
    o.u8(2);                          // version 2
    o.u8(scalar ? 0 : (uint32_t)dims.size());
    o.u8(0);                          // no maximum dimensions
    o.u8(scalar ? 0 : 1);             // scalar or simple
    if (!scalar)
        for (uint64_t d : dims) o.u64(d);
    return o.b;
}

// ---- the tree: sizes, addresses, bytes ------------------------------------------------
struct Msg {
    uint8_t type;
    std::vector<uint8_t> data;
};

static std::vector<uint8_t> attr_msg(const Attr& a) {
    const std::vector<uint8_t> t = type_msg(a.type), sp = space_msg(a.dims, a.scalar);
    Out o;
    o.u8(3);  // version 3
    o.u8(0);
    o.u16((uint32_t)a.name.size() + 1);
    o.u16((uint32_t)t.size());
    o.u16((uint32_t)sp.size());
    o.u8(0);  // ASCII name
    o.raw(a.name.c_str(), a.name.size() + 1);
    o.raw(t.data(), t.size());
    o.raw(sp.data(), sp.size());
    o.raw(a.data.data(), a.data.size());
    return o.b;
}

// the messages of a node; child addresses and the data address are filled in
static std::vector<Msg> messages(const Node& n, const std::vector<uint64_t>& child_addr, uint64_t data_addr) {
    std::vector<Msg> m;
    if (n.is_group) {
        Out li;
        li.u8(0);
        li.u8(0);
        li.u64(UNDEF);  // no fractal heap: links live in this header
        li.u64(UNDEF);  // no name index
        m.push_back({2, li.b});
        // Group Info, version 0, with the link phase change values: every
        // link stays in this header (maximum compact count >= the links)
        Out gi;
        gi.u8(0);
        gi.u8(1);
        gi.u16((uint32_t)std::min<size_t>(65535, std::max<size_t>(8, n.children.size())));
        gi.u16(6);
        m.push_back({10, gi.b});
        for (size_t c = 0; c < n.children.size(); ++c) {
            const std::string& name = n.children[c].name;
            Out l;
            l.u8(1);  // version 1
            l.u8(0);  // 1-byte name length, hard link, ASCII
            l.u8((uint32_t)name.size());
            l.raw(name.data(), name.size());
            l.u64(child_addr[c]);
            m.push_back({6, l.b});
        }
    } else {
        m.push_back({1, space_msg(n.dims, n.scalar)});
        m.push_back({3, type_msg(n.type)});
        m.push_back({5, {3, 0x05}});  // Fill Value v3: allocated early, never written
        Out lay;
        lay.u8(3);  // version 3
        lay.u8(1);  // contiguous
        lay.u64(data_addr);
        lay.u64((uint64_t)n.data.size());
        m.push_back({8, lay.b});
    }
    for (const Attr& a : n.attrs) m.push_back({12, attr_msg(a)});
    return m;
}

static size_t header_size(const std::vector<Msg>& m) {
    size_t s = 4 + 1 + 1 + 4 + 4;  // signature, version, flags, chunk size, checksum
    for (const Msg& x : m) s += 4 + x.data.size();
    return s;
}

static std::vector<uint8_t> header_bytes(const std::vector<Msg>& m) {
    Out o;
    o.raw("OHDR", 4);
    o.u8(2);     // version 2
    o.u8(0x02);  // chunk size in 4 bytes; no times, no creation order
    size_t chunk = 0;
    for (const Msg& x : m) chunk += 4 + x.data.size();
    o.u32((uint32_t)chunk);
    for (const Msg& x : m) {
        o.u8(x.type);
        o.u16((uint32_t)x.data.size());
        o.u8(0);
        o.raw(x.data.data(), x.data.size());
    }
    o.u32(lookup3(o.b.data(), o.b.size(), 0));
    return o.b;
}

int write_file(const char* path, const Node& root, std::string& err) {
    // layout: superblock, every object header (depth first), then the data
    // blocks (8-byte aligned); header sizes do not depend on the addresses
    std::vector<const Node*> order;
    std::function<void(const Node&)> walk = [&](const Node& n) {
        order.push_back(&n);
        for (const Node& c : n.children) walk(c);
    };
    walk(root);
    std::vector<uint64_t> haddr(order.size()), daddr(order.size(), 0);
    const std::vector<uint64_t> zeros_child(64, 0);
    uint64_t pos = 48;
    for (size_t k = 0; k < order.size(); ++k) {
        haddr[k] = pos;
        std::vector<uint64_t> ca(order[k]->children.size(), 0);
        pos += header_size(messages(*order[k], ca, 0));
    }
    for (size_t k = 0; k < order.size(); ++k)
        if (!order[k]->is_group) {
            pos = (pos + 7) & ~(uint64_t)7;
            daddr[k] = pos;
            pos += order[k]->data.size();
        }
    const uint64_t eof = pos;
    std::vector<uint8_t> file(eof, 0);
    // superblock
    Out sb;
    const uint8_t sig[8] = {0x89, 'H', 'D', 'F', '\r', '\n', 0x1a, '\n'};
    sb.raw(sig, 8);
    sb.u8(2);
    sb.u8(8);
    sb.u8(8);
    sb.u8(0);
    sb.u64(0);
    sb.u64(UNDEF);
    sb.u64(eof);
    sb.u64(haddr[0]);
    sb.u32(lookup3(sb.b.data(), sb.b.size(), 0));
    memcpy(file.data(), sb.b.data(), sb.b.size());
    // headers and data
    std::function<size_t(const Node*)> index_of = [&](const Node* p) -> size_t {
        for (size_t k = 0; k < order.size(); ++k)
            if (order[k] == p) return k;
        return 0;
    };
    for (size_t k = 0; k < order.size(); ++k) {
        std::vector<uint64_t> ca;
        for (const Node& c : order[k]->children) ca.push_back(haddr[index_of(&c)]);
        const std::vector<uint8_t> h = header_bytes(messages(*order[k], ca, daddr[k]));
        memcpy(file.data() + haddr[k], h.data(), h.size());
        if (!order[k]->is_group && !order[k]->data.empty())
            memcpy(file.data() + daddr[k], order[k]->data.data(), order[k]->data.size());
    }
    FILE* f = fopen(path, "wb");
    if (!f) {
        err = "cannot open the file for writing";
        return -1;
    }
    const size_t w = fwrite(file.data(), 1, file.size(), f);
    const int cl = fclose(f);
    if (w != file.size() || cl != 0) {
        err = "write failed";
        return -1;
    }
    return 0;
}

// ---- decoder -------------------------------------------------------------------------
namespace {
struct In {
    const std::vector<uint8_t>& b;
    size_t p;
    bool ok = true;
    uint64_t get(int n) {
        if (p + n > b.size()) {
            ok = false;
            return 0;
        }
        uint64_t v = 0;
        for (int i = 0; i < n; ++i) v |= (uint64_t)b[p + i] << (8 * i);
        p += n;
        return v;
    }
};

bool parse_type(In& in, Type& t) {
    const uint32_t cv = (uint32_t)in.get(1);
    const uint32_t b1 = (uint32_t)in.get(1);
    in.get(2);
    t.size = (uint32_t)in.get(4);
    const uint32_t cls = cv & 15;
    if ((cv >> 4) != 1) return false;
    if (cls == 0) {
        t.cls = Type::INT;
        t.is_signed = (b1 & 0x08) != 0;
        in.get(4);
    } else if (cls == 1) {
        t.cls = Type::FLOAT;
        in.get(12);
        if (t.size != 8) return false;
    } else if (cls == 3) {
        t.cls = Type::STRING;
    } else {
        return false;
    }
    return in.ok && (b1 & 1) == 0;  // little-endian only
}

bool parse_space(In& in, std::vector<uint64_t>& dims, bool& scalar) {
    if (in.get(1) != 2) return false;
    const int rank = (int)in.get(1);
    const uint32_t flags = (uint32_t)in.get(1);
    const uint32_t type = (uint32_t)in.get(1);
    scalar = type == 0;
    dims.clear();
    for (int i = 0; i < rank; ++i) dims.push_back(in.get(8));
    if (flags & 1)
        for (int i = 0; i < rank; ++i) in.get(8);
    return in.ok && type <= 1;
}

// Every address and length read from the file is checked against the file's
// size without overflow; each object may be reached once only (the writer
// links every object from one parent), so a file whose links form a cycle or
// reach one object twice is refused rather than walked again.
bool parse_node(const std::vector<uint8_t>& b, uint64_t addr, const std::string& name, Node& n, int depth,
                std::vector<uint64_t>& seen, std::string& err) {
    if (depth > 16) {
        err = "groups nested too deep";
        return false;
    }
    if (addr > b.size() || b.size() - addr < 16 || memcmp(b.data() + addr, "OHDR", 4) != 0) {
        err = "not a version-2 object header at " + std::to_string(addr);
        return false;
    }
    if (std::find(seen.begin(), seen.end(), addr) != seen.end()) {
        err = "an object reached twice";
        return false;
    }
    seen.push_back(addr);
    In in{b, (size_t)addr + 4};
    const uint32_t ver = (uint32_t)in.get(1), flags = (uint32_t)in.get(1);
    if (ver != 2 || (flags & ~3u) != 0) {
        err = "unsupported object header flags";
        return false;
    }
    const uint64_t chunk = in.get(1 << (flags & 3));
    const size_t start = in.p;
    if (!in.ok || chunk > b.size() || b.size() - start < chunk + 4) {
        err = "truncated object header";
        return false;
    }
    const size_t end = start + (size_t)chunk;
    const uint32_t sum = (uint32_t)(b[end] | (b[end + 1] << 8) | (b[end + 2] << 16) | ((uint32_t)b[end + 3] << 24));
    if (sum != lookup3(b.data() + addr, end - addr, 0)) {
        err = "object header checksum mismatch";
        return false;
    }
    n.name = name;
    n.is_group = false;
    uint64_t data_addr = UNDEF, data_size = 0;
    bool have_layout = false;
    std::vector<std::pair<std::string, uint64_t>> links;
    while (in.p + 4 <= end) {
        const uint32_t type = (uint32_t)in.get(1);
        const uint32_t size = (uint32_t)in.get(2);
        in.get(1);
        const size_t mend = in.p + size;
        if (mend > end) {
            err = "message past the header";
            return false;
        }
        In m{b, in.p};
        if (type == 2) {
            n.is_group = true;
        } else if (type == 6) {
            if (m.get(1) != 1 || m.get(1) != 0) {
                err = "unsupported link message";
                return false;
            }
            const size_t len = (size_t)m.get(1);
            if (m.p + len + 8 > mend) {
                err = "bad link message";
                return false;
            }
            std::string ln(reinterpret_cast<const char*>(b.data() + m.p), len);
            m.p += len;
            links.push_back({ln, m.get(8)});
        } else if (type == 1) {
            if (!parse_space(m, n.dims, n.scalar)) {
                err = "unsupported dataspace";
                return false;
            }
        } else if (type == 3) {
            if (!parse_type(m, n.type)) {
                err = "unsupported datatype";
                return false;
            }
        } else if (type == 8) {
            if (m.get(1) != 3 || m.get(1) != 1) {
                err = "only contiguous storage is read";
                return false;
            }
            data_addr = m.get(8);
            data_size = m.get(8);
            have_layout = true;
        } else if (type == 12) {
            Attr a;
            if (m.get(1) != 3) {
                err = "unsupported attribute message";
                return false;
            }
            m.get(1);
            const size_t nl = (size_t)m.get(2), tl = (size_t)m.get(2), sl = (size_t)m.get(2);
            m.get(1);
            if (nl == 0 || m.p + nl + tl + sl > mend) {
                err = "bad attribute message";
                return false;
            }
            a.name.assign(reinterpret_cast<const char*>(b.data() + m.p), nl - 1);
            m.p += nl;
            In tm{b, m.p};
            if (!parse_type(tm, a.type)) {
                err = "unsupported attribute datatype";
                return false;
            }
            m.p += tl;
            In sm{b, m.p};
            if (!parse_space(sm, a.dims, a.scalar)) {
                err = "unsupported attribute dataspace";
                return false;
            }
            m.p += sl;
            a.data.assign(b.begin() + m.p, b.begin() + mend);
            n.attrs.push_back(a);
        }
        in.p = mend;
    }
    if (n.is_group) {
        for (const auto& l : links) {
            Node c;
            if (!parse_node(b, l.second, l.first, c, depth + 1, seen, err)) return false;
            n.children.push_back(std::move(c));
        }
    } else {
        if (!have_layout || data_addr > b.size() || data_size > b.size() - data_addr) {
            err = "dataset without readable data";
            return false;
        }
        n.data.assign(b.begin() + data_addr, b.begin() + data_addr + data_size);
    }
    return true;
}
}  // namespace

int read_file(const char* path, Node& root, std::string& err) {
    FILE* f = fopen(path, "rb");
    if (!f) {
        err = "cannot open the file";
        return -1;
    }
    std::vector<uint8_t> b;
    uint8_t buf[1 << 16];
    size_t r;
    while ((r = fread(buf, 1, sizeof(buf), f)) > 0) b.insert(b.end(), buf, buf + r);
    fclose(f);
    const uint8_t sig[8] = {0x89, 'H', 'D', 'F', '\r', '\n', 0x1a, '\n'};
    if (b.size() < 48 || memcmp(b.data(), sig, 8) != 0 || b[8] != 2 || b[9] != 8 || b[10] != 8) {
        err = "not an HDF5 file with a version-2 superblock";
        return -1;
    }
    const uint32_t sum = (uint32_t)(b[44] | (b[45] << 8) | (b[46] << 16) | ((uint32_t)b[47] << 24));
    if (sum != lookup3(b.data(), 44, 0)) {
        err = "superblock checksum mismatch";
        return -1;
    }
    In in{b, 36};
    const uint64_t root_addr = in.get(8);
    std::vector<uint64_t> seen;
    return parse_node(b, root_addr, "", root, 0, seen, err) ? 0 : -1;
}

// ---- tree helpers ----------------------------------------------------------------------
Node& Node::group(const std::string& n) {
    for (Node& c : children)
        if (c.name == n) return c;
    Node c;
    c.name = n;
    c.is_group = true;
    children.push_back(c);
    return children.back();
}

const Node* Node::find(const std::string& path) const {
    const Node* cur = this;
    size_t p = 0;
    while (p < path.size()) {
        size_t q = path.find('/', p);
        if (q == std::string::npos) q = path.size();
        const std::string part = path.substr(p, q - p);
        p = q + 1;
        if (part.empty()) continue;
        const Node* next = nullptr;
        for (const Node& c : cur->children)
            if (c.name == part) next = &c;
        if (!next) return nullptr;
        cur = next;
    }
    return cur;
}

}  // namespace h5
}  // namespace espp
