// H5MD files without an HDF5 library: a small HDF5 encoder/decoder (h5md.cpp)
// and the H5MD layout of a handle's state (h5md_layout.cpp).  Host code only.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace espp {
namespace h5 {

struct Type {
    enum Cls { INT, FLOAT, STRING } cls = FLOAT;
    uint32_t size = 8;      // bytes of one element (a fixed-length string: its length)
    bool is_signed = true;  // fixed-point types
};

struct Attr {
    std::string name;
    Type type;
    std::vector<uint64_t> dims;
    bool scalar = false;
    std::vector<uint8_t> data;  // little-endian elements
};

// A group (children, attributes) or a dataset (type, shape, contiguous data).
struct Node {
    std::string name;
    bool is_group = true;
    std::vector<Node> children;
    std::vector<Attr> attrs;
    Type type;
    std::vector<uint64_t> dims;
    bool scalar = false;
    std::vector<uint8_t> data;
    // the child group of that name, created if absent (the reference is
    // valid until the next child is added)
    Node& group(const std::string& n);
    // a descendant by a '/'-separated path, or nullptr
    const Node* find(const std::string& path) const;
};

// Bob Jenkins' lookup3 hashlittle, the checksum of HDF5 metadata.
uint32_t lookup3(const uint8_t* key, size_t length, uint32_t initval);
// 0 on success, else -1 with a message in err.
int write_file(const char* path, const Node& root, std::string& err);
int read_file(const char* path, Node& root, std::string& err);

}  // namespace h5

// The state a handle keeps in an H5MD file (particle arrays in id order).
struct H5mdReplica {
    double box[3];
    int64_t n = 0;
    std::vector<double> x, v;      // n x 3
    std::vector<int32_t> img;      // n x 3
    std::vector<double> f;         // n x 3 stored total force, or empty
    std::vector<int32_t> species;  // n
    std::vector<int64_t> bonds;    // n_bonds x 2 local ids
    uint64_t seed = 0;
};
struct H5mdState {
    int64_t step = 0;
    double time = 0.0;
    int32_t precision = 0;
    int32_t lees_edwards = 0;
    double shear_rate = 0.0;
    std::vector<H5mdReplica> reps;
};

int h5md_write(const char* path, const H5mdState& st, std::string& err);
int h5md_read(const char* path, H5mdState& st, std::string& err);

}  // namespace espp
