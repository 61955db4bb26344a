"""A small HDF5 reader for the tests, written from the HDF5 file-format
specification and independent of the library's encoder: superblock version 2,
version-2 object headers (every flag of the header prefix honoured), groups
held as Link messages, datasets with contiguous or compact storage,
attributes (message version 3), fixed-point, IEEE floating-point and
fixed-length string datatypes.  Every checksum (Jenkins lookup3 hashlittle,
initial value 0) is verified; a mismatch raises."""
import struct

import numpy as np

UNDEF = 0xFFFFFFFFFFFFFFFF
SIGNATURE = b"\x89HDF\r\n\x1a\n"


def hashlittle(data: bytes, initval: int = 0) -> int:
    """Bob Jenkins' lookup3 hashlittle on a byte string (little-endian reads)."""
    M = 0xFFFFFFFF

    def rot(x, k):
        return ((x << k) | (x >> (32 - k))) & M

    n = len(data)
    a = b = c = (0xDEADBEEF + n + initval) & M
    i = 0
    while n - i > 12:
        a = (a + int.from_bytes(data[i:i + 4], "little")) & M
        b = (b + int.from_bytes(data[i + 4:i + 8], "little")) & M
        c = (c + int.from_bytes(data[i + 8:i + 12], "little")) & M
        a = (a - c) & M; a ^= rot(c, 4); c = (c + b) & M
        b = (b - a) & M; b ^= rot(a, 6); a = (a + c) & M
        c = (c - b) & M; c ^= rot(b, 8); b = (b + a) & M
        a = (a - c) & M; a ^= rot(c, 16); c = (c + b) & M
        b = (b - a) & M; b ^= rot(a, 19); a = (a + c) & M
        c = (c - b) & M; c ^= rot(b, 4); b = (b + a) & M
        i += 12
    tail = data[i:]
    if len(tail) == 0:
        return c
    pad = tail + bytes(12 - len(tail))
    a = (a + int.from_bytes(pad[0:4], "little")) & M
    b = (b + int.from_bytes(pad[4:8], "little")) & M
    c = (c + int.from_bytes(pad[8:12], "little")) & M
    c ^= b; c = (c - rot(b, 14)) & M
    a ^= c; a = (a - rot(c, 11)) & M
    b ^= a; b = (b - rot(a, 25)) & M
    c ^= b; c = (c - rot(b, 16)) & M
    a ^= c; a = (a - rot(c, 4)) & M
    b ^= a; b = (b - rot(a, 14)) & M
    c ^= b; c = (c - rot(b, 24)) & M
    return c


class Group:
    def __init__(self):
        self.attrs = {}
        self.children = {}

    def __getitem__(self, path):
        node = self
        for part in path.strip("/").split("/"):
            node = node.children[part]
        return node


class Dataset:
    def __init__(self, value, attrs):
        self.value = value
        self.attrs = attrs


def _u(buf, off, n):
    return int.from_bytes(buf[off:off + n], "little")


def _datatype(buf, off):
    """(numpy dtype, bytes consumed) of a datatype message at off."""
    cv = buf[off]
    cls, ver = cv & 15, cv >> 4
    bits = buf[off + 1] | (buf[off + 2] << 8) | (buf[off + 3] << 16)
    size = _u(buf, off + 4, 4)
    assert ver in (1, 2, 3), "datatype version"
    if cls == 0:       # fixed-point: byte order bit 0, signed bit 3
        assert bits & 1 == 0, "big-endian integers"
        signed = bool(bits & 8)
        return np.dtype(("<i%d" if signed else "<u%d") % size), 8 + 4
    if cls == 1:       # floating point: IEEE layout checked field by field
        assert bits & 1 == 0 and size in (4, 8)
        bit_off, prec, eloc, esz, mloc, msz = struct.unpack_from("<HHBBBB", buf, off + 8)
        bias = _u(buf, off + 16, 4)
        ieee = {4: (32, 23, 8, 0, 23, 127), 8: (64, 52, 11, 0, 52, 1023)}[size]
        assert (bit_off, prec, eloc, esz, mloc, msz, bias) == (0,) + ieee, "not an IEEE float"
        assert (bits >> 8) & 0xFF == 8 * size - 1, "sign bit position"
        return np.dtype("<f%d" % size), 8 + 12
    if cls == 3:       # fixed-length string
        return np.dtype("S%d" % size), 8
    raise AssertionError("datatype class %d" % cls)


def _dataspace(buf, off):
    ver = buf[off]
    if ver == 2:
        rank, flags, kind = buf[off + 1], buf[off + 2], buf[off + 3]
        p = off + 4
        dims = [_u(buf, p + 8 * k, 8) for k in range(rank)]
        return (() if kind == 0 else tuple(dims)), kind
    if ver == 1:
        rank, flags = buf[off + 1], buf[off + 2]
        p = off + 8
        dims = [_u(buf, p + 8 * k, 8) for k in range(rank)]
        return tuple(dims), 1
    raise AssertionError("dataspace version %d" % ver)


def _attribute(buf, off):
    ver = buf[off]
    assert ver == 3, "attribute message version"
    nlen, tlen, slen = struct.unpack_from("<HHH", buf, off + 2)
    p = off + 9
    name = buf[p:p + nlen].split(b"\0")[0].decode()
    p += nlen
    dt, _ = _datatype(buf, p)
    p += tlen
    shape, kind = _dataspace(buf, p)
    p += slen
    count = int(np.prod(shape)) if shape else 1
    val = np.frombuffer(bytes(buf[p:p + count * dt.itemsize]), dtype=dt).reshape(shape)
    return name, val


def _object(buf, addr, depth=0):
    assert depth < 32
    assert buf[addr:addr + 4] == b"OHDR", "object header signature"
    ver, flags = buf[addr + 4], buf[addr + 5]
    assert ver == 2
    p = addr + 6
    if flags & 0x20:   # access, modification, change, birth times
        p += 16
    if flags & 0x10:   # attribute phase change values
        p += 4
    width = 1 << (flags & 3)
    chunk = _u(buf, p, width)
    p += width
    end = p + chunk
    assert _u(buf, end, 4) == hashlittle(bytes(buf[addr:end])), "object header checksum"
    order = bool(flags & 0x04)
    attrs, links = {}, []
    dtype = shape = layout = None
    group = False
    while end - p >= (6 if order else 4):
        mtype, msize = buf[p], _u(buf, p + 1, 2)
        p += 4 + (2 if order else 0)
        body = p
        if mtype in (2, 10):       # link info, group info
            group = True
        elif mtype == 6:           # link
            lflags = buf[body + 1]
            q = body + 2
            ltype = 0
            if lflags & 0x08:
                ltype = buf[q]; q += 1
            if lflags & 0x04:
                q += 8
            if lflags & 0x10:
                q += 1
            lw = 1 << (lflags & 3)
            ln = _u(buf, q, lw); q += lw
            name = bytes(buf[q:q + ln]).decode(); q += ln
            assert ltype == 0, "only hard links"
            links.append((name, _u(buf, q, 8)))
            group = True
        elif mtype == 1:
            shape, _ = _dataspace(buf, body)
        elif mtype == 3:
            dtype, _ = _datatype(buf, body)
        elif mtype == 8:           # data layout, version 3
            assert buf[body] == 3
            cls = buf[body + 1]
            if cls == 1:
                layout = ("contiguous", _u(buf, body + 2, 8), _u(buf, body + 10, 8))
            elif cls == 0:
                sz = _u(buf, body + 2, 2)
                layout = ("compact", body + 4, sz)
            else:
                raise AssertionError("chunked storage")
        elif mtype == 12:
            name, val = _attribute(buf, body)
            attrs[name] = val
        p = body + msize
    if group:
        g = Group()
        g.attrs = attrs
        for name, a in links:
            g.children[name] = _object(buf, a, depth + 1)
        return g
    assert dtype is not None and shape is not None and layout is not None
    _, start, size = layout
    count = int(np.prod(shape)) if shape else 1
    assert size == count * dtype.itemsize, "data size differs from the shape"
    assert start != UNDEF and start + size <= len(buf)
    val = np.frombuffer(bytes(buf[start:start + size]), dtype=dtype).reshape(shape)
    return Dataset(val, attrs)


def read(path):
    """The root group of an HDF5 file with a version-2 superblock."""
    buf = open(path, "rb").read()
    assert buf[:8] == SIGNATURE, "HDF5 signature"
    assert buf[8] in (2, 3), "superblock version"
    so, sl = buf[9], buf[10]
    assert so == 8 and sl == 8
    assert _u(buf, 44, 4) == hashlittle(buf[:44]), "superblock checksum"
    base, ext, eof, root = struct.unpack_from("<QQQQ", buf, 12)
    assert base == 0 and eof == len(buf), "end-of-file address"
    return _object(buf, root)
