"""The headless figure writer of the fixed-omega comparison (Examples 5.5,
5.9, 5.10): the PNG encoder is read back with a decoder written here from
the PNG format (signature, length-tag-data-CRC chunks, IHDR, zlib IDAT with a
filter byte per row), and the plot helpers keep every drawn pixel inside its
panel."""
import os
import shutil
import struct
import zlib

import numpy as np
import pytest

from paper_2609_18177_b300 import figures as F

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def read_png(path):
    data = open(path, "rb").read()
    assert data[:8] == b"\x89PNG\r\n\x1a\n"
    pos, chunks = 8, []
    while pos < len(data):
        (n,) = struct.unpack(">I", data[pos:pos + 4])
        tag, body = data[pos + 4:pos + 8], data[pos + 8:pos + 8 + n]
        (crc,) = struct.unpack(">I", data[pos + 8 + n:pos + 12 + n])
        assert crc == zlib.crc32(tag + body) & 0xFFFFFFFF, tag
        chunks.append((tag, body))
        pos += 12 + n
    assert [t for t, _ in chunks] == [b"IHDR", b"IDAT", b"IEND"]
    w, h, depth, ctype, comp, filt, inter = struct.unpack(">IIBBBBB", chunks[0][1])
    assert (depth, ctype, comp, filt, inter) == (8, 2, 0, 0, 0)  # 8-bit RGB, no interlace
    raw = zlib.decompress(chunks[1][1])
    assert len(raw) == h * (1 + 3 * w)
    rows = [raw[r * (1 + 3 * w):(r + 1) * (1 + 3 * w)] for r in range(h)]
    assert all(row[0] == 0 for row in rows)  # filter type 0 (None) on every row
    return np.frombuffer(b"".join(row[1:] for row in rows), dtype=np.uint8).reshape(h, w, 3)


@pytest.fixture
def outdir():
    d = os.path.join(ROOT, "_build", "figures_png")  # git-ignored build folder
    shutil.rmtree(d, ignore_errors=True)
    os.makedirs(d)
    yield d
    shutil.rmtree(d, ignore_errors=True)


def test_png_roundtrip(outdir):
    rng = np.random.default_rng(4)
    img = rng.integers(0, 256, size=(37, 53, 3), dtype=np.uint8)
    path = os.path.join(outdir, "r.png")
    F.write_png(path, img)
    assert np.array_equal(read_png(path), img)


def test_panel_lines_stay_inside_and_hit_the_ends(outdir):
    img = np.full((120, 200, 3), 255, dtype=np.uint8)
    p = F.Panel(img, 10, 20, 150, 80, xlim=(0.0, 1.0), ylim=(-1.0, 1.0))
    x = np.linspace(0.0, 1.0, 50)
    p.line(x, 3.0 * np.sin(6 * x), F.BLUE, thick=3)  # overshoots the y range: clipped
    blue = np.all(img == np.array(F.BLUE, dtype=np.uint8), axis=2)
    ys, xs = np.nonzero(blue)
    assert xs.min() >= 10 and xs.max() <= 10 + 150 - 1 and ys.min() >= 20 and ys.max() <= 20 + 80 - 1
    assert blue[:, 10].any() and blue[:, 159].any()  # the curve spans the panel
    path = os.path.join(outdir, "p.png")
    F.write_png(path, img)
    assert np.array_equal(read_png(path), img)


def test_limits_and_heat():
    lo, hi = F.limits(np.array([0.0, 1.0]), np.array([2.0, np.nan]))
    assert lo == pytest.approx(-0.16) and hi == pytest.approx(2.16)
    assert F.limits(np.array([3.0, 3.0])) == (pytest.approx(3.0 - 0.08), pytest.approx(3.0 + 0.08))
    img = np.zeros((4, 6, 3), dtype=np.uint8)
    field = np.array([[0.0, 1.0], [0.5, 2.0]])  # row 0 is drawn at the bottom
    F.heat(img, 1, 1, field, 0.0, 1.0)
    assert img[2, 1, 0] == 255 and img[2, 2, 0] == 0      # bottom row: 0 -> white, 1 -> black
    assert img[1, 1, 0] == 127 and img[1, 2, 0] == 0      # top row: 0.5 -> grey, 2 clipped to black
