"""A minimal HDF5 writer for the tests, written from the HDF5 file-format
specification and independent of the library's encoder: a version-2
superblock, version-2 object headers, groups held as Link Info, Group Info
and Link messages, datasets with a version-2 dataspace, version-1 datatype
and contiguous layout (version 3), attributes (message version 3).  It lays
objects out child first, so a parent's links hold known addresses, and lets a
test plant malformed fields (shapes, addresses, links) on purpose."""
import struct

from _h5read import hashlittle

UNDEF = 0xFFFFFFFFFFFFFFFF
SIGNATURE = b"\x89HDF\r\n\x1a\n"


def t_int(size, signed=True):
    # class 0 (fixed-point), version 1; bit field: little-endian, bit 3 signed;
    # properties: bit offset 0, precision 8 * size
    return bytes([0x10, 0x08 if signed else 0x00, 0, 0]) + struct.pack("<IHH", size, 0, 8 * size)


def t_f64():
    # class 1 (floating point), version 1; bit field: little-endian, implied
    # mantissa bit (normalisation 2), sign at bit 63; IEEE binary64 layout
    return bytes([0x11, 0x20, 63, 0]) + struct.pack("<IHHBBBBI", 8, 0, 64, 52, 11, 0, 52, 1023)


def space(dims, scalar=False):
    return bytes([2, 0 if scalar else len(dims), 0, 0 if scalar else 1]) + b"".join(
        struct.pack("<Q", d) for d in ([] if scalar else dims))


def msg(mtype, body):
    return struct.pack("<BHB", mtype, len(body), 0) + body


def attribute(name, dtype, dims, data, scalar=False):
    nm = name.encode() + b"\0"
    ds = space(dims, scalar)
    return msg(12, bytes([3, 0]) + struct.pack("<HHH", len(nm), len(dtype), len(ds)) + bytes([0]) + nm + dtype
               + ds + data)


class Dataset:
    def __init__(self, dtype, dims, data, attrs=(), addr=None, size=None):
        self.dtype, self.dims, self.data, self.attrs = dtype, list(dims), data, list(attrs)
        self.addr, self.size = addr, size  # planted layout fields (None: where the data lie)


class Group:
    def __init__(self, children=None, attrs=(), links=()):
        self.children = dict(children or {})
        self.attrs = list(attrs)
        # extra links planted as they are: (name, address), (name, "self") for
        # a link to this group, (name, node) for a node already written
        self.links = list(links)


class File:
    def __init__(self):
        self.buf = bytearray(48)
        self.where = {}

    def _put(self, b):
        addr = len(self.buf)
        self.buf += b
        return addr

    def _header(self, messages):
        body = b"".join(messages)
        if len(body) < 256:
            flags, size = 0, struct.pack("<B", len(body))
        elif len(body) < 65536:
            flags, size = 1, struct.pack("<H", len(body))
        else:
            flags, size = 2, struct.pack("<I", len(body))
        h = b"OHDR" + bytes([2, flags]) + size + body
        return self._put(h + struct.pack("<I", hashlittle(bytes(h))))

    def add(self, node):
        if isinstance(node, Dataset):
            daddr = self._put(node.data)
            addr = daddr if node.addr is None else node.addr
            size = len(node.data) if node.size is None else node.size
            msgs = [msg(1, space(node.dims)), msg(3, node.dtype),
                    msg(8, bytes([3, 1]) + struct.pack("<QQ", addr, size))]
            self.where[id(node)] = self._header(msgs + node.attrs)
            return self.where[id(node)]
        links = [(name, self.add(child)) for name, child in node.children.items()]
        for name, a in node.links:
            links.append((name, a if isinstance(a, int) else self.where[id(a)] if a != "self" else None))
        msgs = [msg(2, bytes([0, 0]) + struct.pack("<QQ", UNDEF, UNDEF)), msg(10, bytes([0, 0]))]
        # the header goes at the end of the buffer: a link to "self" points there
        msgs += [msg(6, bytes([1, 0, len(name.encode())]) + name.encode()
                     + struct.pack("<Q", len(self.buf) if a is None else a)) for name, a in links]
        self.where[id(node)] = self._header(msgs + node.attrs)
        return self.where[id(node)]

    def bytes(self, root, root_addr=None):
        addr = self.add(root)
        sb = bytearray(SIGNATURE + bytes([2, 8, 8, 0]))
        sb += struct.pack("<QQQQ", 0, UNDEF, len(self.buf), addr if root_addr is None else root_addr)
        sb += struct.pack("<I", hashlittle(bytes(sb)))
        self.buf[:48] = sb
        return bytes(self.buf)
