"""CPU checks of the PNG writer used for headless image export: a hand-written decoder reads the bytes back."""
import struct
import zlib

import numpy as np

from paper_2501_12750_gb300.export import png_bytes, write_png


def decode_png(b: bytes) -> np.ndarray:
    """Minimal decoder for what png_bytes writes: 8-bit RGBA, filter type 0 rows, CRC-checked chunks."""
    assert b[:8] == b"\x89PNG\r\n\x1a\n"
    pos, idat, W = 8, b"", None
    while pos < len(b):
        (n,) = struct.unpack(">I", b[pos:pos + 4])
        tag, data = b[pos + 4:pos + 8], b[pos + 8:pos + 8 + n]
        (crc,) = struct.unpack(">I", b[pos + 8 + n:pos + 12 + n])
        assert crc == zlib.crc32(tag + data) & 0xFFFFFFFF
        if tag == b"IHDR":
            W, H, depth, ctype, comp, filt, inter = struct.unpack(">IIBBBBB", data)
            assert (depth, ctype, comp, filt, inter) == (8, 6, 0, 0, 0)
        elif tag == b"IDAT":
            idat += data
        pos += 12 + n
    raw = np.frombuffer(zlib.decompress(idat), np.uint8).reshape(H, 1 + 4 * W)
    assert (raw[:, 0] == 0).all()
    return raw[:, 1:].reshape(H, W, 4)


def test_png_round_trip_random_image():
    a = np.random.default_rng(3).integers(0, 256, (37, 53, 4), dtype=np.uint8)
    np.testing.assert_array_equal(decode_png(png_bytes(a)), a)


def test_png_file_and_transparent_background(tmp_path):
    a = np.zeros((8, 5, 4), np.uint8)
    a[..., :3] = 255
    a[2:5, 1:3] = (10, 20, 30, 255)
    p = tmp_path / "x.png"
    write_png(str(p), a)
    back = decode_png(p.read_bytes())
    np.testing.assert_array_equal(back, a)
    assert (back[..., 3] == 0).sum() == 40 - 6
