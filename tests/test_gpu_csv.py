"""CSV extract kernel against the oracle's parser: parsed rows bit-exact, the same malformed
count, then the whole path on the parsed rows."""
import os

import numpy as np
import pytest

import cvgen
from parity import compare, exact

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def gpu_csv(text, device=False, materialize=True):
    import torch

    import paper_2305_07454_b300 as P

    if isinstance(text, (bytes, bytearray)):
        text = np.frombuffer(bytes(text), dtype=np.uint8).copy()
    t = torch.from_numpy(np.ascontiguousarray(text))
    if device:
        t = t.cuda()
    with P.Pipeline(materialize_points=int(materialize)) as p:
        p.extract_csv(t)
        x = p.extracted()
        p.transform()
        p.load()
        r = p.results()
    return x, r


def check_parse(orc, text, **kw):
    want, n_lines, n_bad = orc.parse_csv(text)
    got, r = gpu_csv(text, **kw)
    assert r["counters"]["n_in"] == n_lines, (r["counters"]["n_in"], n_lines)
    for k in ("jid", "ts", "lat", "lon", "speed", "heading"):
        exact("parsed " + k, got[k], want[k])
    o = orc.run(want)
    assert o["counters"]["n_in"] == n_lines and o["counters"]["n_malformed"] >= n_bad
    compare(r, o, points=o["counters"]["n_valid"] > 0)
    return r


def test_table1_golden(orc):
    text = open(os.path.join(GOLDEN, "table1.csv"), "rb").read()
    r = check_parse(orc, text)
    assert r["counters"]["n_cells"] == 3 and list(r["cells"]["key"]) == [70381134, 70689335, 70691345]


def test_small_day_with_malformed_rows(orc, small_day):
    text, injected = cvgen.to_csv(small_day, seed=3, malformed_frac=0.02)
    r = check_parse(orc, text)
    assert r["counters"]["n_malformed"] == injected
    check_parse(orc, text, device=True)


def test_line_edge_cases(orc):
    rows = [
        b"1,1620520000000,37.5,-92.5,10.5,90",
        b"1,1620520000500,37.500001,-92.500001,11,90.5\r",  # CRLF
        b"",  # empty line
        b"2,1620520000000,-0,-0.0,-0,0",  # negative zeros
        b"2,1620520001000,90,180,1.5,1",  # range edges
        b"2,1620520002000,90.0000001,180,1,1",  # out of range
        b"3,1620520000000,37.123456789012345,-92,1,1",  # 17 digits
        b"3,1620520000000,37.12345678901234,-92,1,1",  # 16 digits
        b"3,1620520000000,7.12345678901234,-92,1,1",  # 15 digits
        b"3,1620520000000,1e5,-92,1,1",
        b"3,1620520000000,.5,-92,1,1",
        b"3,1620520000000,5.,-92,1,1",
        b"3,1620520000000,+5,-92,1,1",
        b"3,1620520000000,5,-92,1,1,",  # extra empty field
        b"3,1620520000000,5,-92,1",  # missing field
        b"3,,5,-92,1,1",  # empty integer
        b"-,1620520000000,5,-92,1,1",
        b"1234567890123456789,1620520000000,5,-92,1,1",  # 19-digit id
        b"-123456789012345678,1620520003000,5,-92,1,1",
        b"4,1620520000000,nan,-92,1,1",
        b"4,16205200x0000,5,-92,1,1",
        b"5," + b"9" * 3000 + b",5,-92,1,1",  # a very long line
        b"6,1620520009000,38.5,-91.5,0.25,359.9",
    ]
    text = b"\n".join(rows)  # no trailing newline
    check_parse(orc, text)
    check_parse(orc, text + b"\n")
    check_parse(orc, b"\n\n\n")
    check_parse(orc, b"")


def test_tiles_of_tiny_lines_and_long_lines(orc):
    rng = np.random.default_rng(5)
    parts = []
    for i in range(6000):
        r = rng.random()
        if r < 0.4:
            parts.append(b"")  # empty lines: very many line starts per tile
        elif r < 0.45:
            parts.append(b"x" * int(rng.integers(500, 5000)))  # long garbage lines cross tiles
        else:
            lat = f"{rng.uniform(36, 40.6):.{int(rng.integers(1, 8))}f}"
            lon = f"{rng.uniform(-95.8, -89.1):.{int(rng.integers(1, 8))}f}"
            parts.append(f"{int(rng.integers(0, 50))},{1620518400000 + int(rng.integers(0, 86_400_000))},"
                         f"{lat},{lon},{rng.uniform(0, 130):.2f},{rng.uniform(0, 360):.1f}".encode())
    check_parse(orc, b"\n".join(parts) + b"\n")


def test_decimal_conversion_is_correctly_rounded(orc):
    """Random decimals of 1-15 digits: the GPU's exact integer conversion against CPython's
    correctly rounded float() (binary64 for lat/lon, then float32 for speed/heading)."""
    rng = np.random.default_rng(9)
    lines, lats, spds = [], [], []
    for i in range(20000):
        ip = int(rng.integers(0, 90))
        nf = int(rng.integers(0, 14 if ip >= 10 else 15))
        frac = "".join(str(d) for d in rng.integers(0, 10, nf))
        lat = (("-" if rng.random() < 0.5 else "") + str(ip) + ("." + frac if nf else ""))
        nd = int(rng.integers(1, 16))
        k = int(rng.integers(0, nd + 1))
        if k == nd == 15:  # "0." + 15 digits would be 16 digits
            k = 14
        digits = "".join(str(d) for d in rng.integers(0, 10, nd))
        spd = (digits[: nd - k] or "0") + ("." + digits[nd - k:] if k else "")
        lines.append(f"{i},{1620518400000 + i},{lat},-92.5,{spd},{spd}".encode())
        lats.append(float(lat))
        spds.append(float(spd))
    text = b"\n".join(lines)
    want, _, bad = orc.parse_csv(text)
    assert bad == 0
    got, _ = gpu_csv(text, materialize=False)
    exact("lat", got["lat"], want["lat"])
    exact("speed", got["speed"], want["speed"])
    exact("heading", got["heading"], want["heading"])
    assert np.array_equal(got["lat"], np.array(lats))
    assert np.array_equal(got["speed"], np.array(spds).astype(np.float32))


def test_decimal_edge_values(orc):
    """Decimals at the ends of the grammar: 14 fraction digits after a 0 (the widest shift),
    15 integer digits (the exact integer path), zeros with fraction digits, negative zero,
    trailing zeros, 16-digit and malformed fields; each against CPython's correctly rounded
    float()."""
    vals = ["0.00000000000001", "0.00000000000009", "0.10000000000000", "-0.00000000000001",
            "999999999999999", "99999999999999.9", "0.99999999999999", "1.00000000000000",
            "0.0", "-0.0", "0.1", "0.2", "0.3", "2.675", "1.005", "179.999999999999",
            "123456789.012345", "0.5", "1.5", "2.5", "4503599627370.49", "9007199254740.99",
            "16777216.5", "16777217", "3.40282346638528", "0.000000000000001", "1e3", "1.2.3"]
    lines = [f"{i},{1620518400000 + i},37.5,{v if _num(v) is not None and abs(_num(v)) <= 180 else '-92.5'},"
             f"{v},{v}".encode() for i, v in enumerate(vals)]
    text = b"\n".join(lines)
    want, _, _ = orc.parse_csv(text)
    got, _ = gpu_csv(text, materialize=False)
    for k in ("lon", "speed", "heading"):
        exact(k, got[k], want[k])
    for i, v in enumerate(vals):
        if _num(v) is None:
            assert np.isnan(got["speed"][i]), v
        else:
            assert got["speed"][i] == np.float32(float(v)) and np.signbit(got["speed"][i]) == v.startswith("-"), v


def _num(v):
    """The value of a field of the decimal grammar (at most 15 digits), else None."""
    import re

    if not re.fullmatch(r"-?[0-9]+(\.[0-9]+)?", v) or sum(ch.isdigit() for ch in v) > 15:
        return None
    return float(v)
