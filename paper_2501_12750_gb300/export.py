"""PNG files from exported RGBA8 images (host side; standard library only).

The renderer packs its planes into interleaved 8-bit RGBA on the GPU
(``Renderer.export_rgba8``); this module writes such an array as a PNG
(colour type 6: 8-bit RGBA, straight alpha), the headless form of the
paper's image export.
"""
from __future__ import annotations

import struct
import zlib

import numpy as np


def _chunk(tag: bytes, data: bytes) -> bytes:
    return struct.pack(">I", len(data)) + tag + data + struct.pack(">I", zlib.crc32(tag + data) & 0xFFFFFFFF)


def png_bytes(rgba: np.ndarray, level: int = 6) -> bytes:
    """PNG encoding of an (H, W, 4) uint8 array: filter type 0 on every row, one zlib stream."""
    a = np.ascontiguousarray(rgba, dtype=np.uint8)
    if a.ndim != 3 or a.shape[2] != 4:
        raise ValueError("expected an (H, W, 4) uint8 array")
    H, W = a.shape[0], a.shape[1]
    rows = np.zeros((H, 1 + 4 * W), np.uint8)  # leading 0 = filter "None"
    rows[:, 1:] = a.reshape(H, 4 * W)
    ihdr = struct.pack(">IIBBBBB", W, H, 8, 6, 0, 0, 0)
    return (b"\x89PNG\r\n\x1a\n" + _chunk(b"IHDR", ihdr) + _chunk(b"IDAT", zlib.compress(rows.tobytes(), level)) +
            _chunk(b"IEND", b""))


def write_png(path: str, rgba: np.ndarray, level: int = 6) -> None:
    with open(path, "wb") as f:
        f.write(png_bytes(rgba, level))
