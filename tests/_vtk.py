"""A small reader of the VTK XML files the library writes (one piece, raw
appended data, UInt64 headers), for the tests."""
import re
import xml.etree.ElementTree as ET

import numpy as np

_TYPES = {"Float32": np.float32, "Float64": np.float64}


def read(path):
    """Returns (kind, extent (nx, ny, nz), attrs of the dataset element,
    {name: array}) with point-data arrays shaped (nz, ny, nx) and Points
    shaped (nz, ny, nx, 3)."""
    raw = open(path, "rb").read()
    mark = raw.index(b'<AppendedData encoding="raw">')
    start = raw.index(b"_", mark) + 1
    tail = raw.rindex(b"</AppendedData>")
    header = raw[:start - 1].decode() + "</AppendedData></VTKFile>"
    root = ET.fromstring(header)
    assert root.get("byte_order") == "LittleEndian" and root.get("header_type") == "UInt64"
    kind = root.get("type")
    ds = root.find(kind)
    ext = [int(v) for v in ds.get("WholeExtent").split()]
    nx, ny, nz = ext[1] + 1, ext[3] + 1, ext[5] + 1
    out = {}
    for da in root.iter("DataArray"):
        assert da.get("format") == "appended"
        off = start + int(da.get("offset"))
        nbytes = int(np.frombuffer(raw, dtype="<u8", count=1, offset=off)[0])
        dt = _TYPES[da.get("type")]
        a = np.frombuffer(raw, dtype=dt, count=nbytes // np.dtype(dt).itemsize, offset=off + 8)
        comps = int(da.get("NumberOfComponents", "1"))
        shape = (nz, ny, nx) if comps == 1 else (nz, ny, nx, comps)
        out[da.get("Name")] = a.reshape(shape)
    return kind, (nx, ny, nz), dict(ds.attrib), out
