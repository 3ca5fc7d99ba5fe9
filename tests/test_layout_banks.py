"""Shared-memory bank analysis of the FP32 stage-kernel layouts (StageGeom in
csrc/stage_kernel.cuh): x-lines vector-read by quarter- or half-warps, y / z lines read one node per
thread, the stage update's quads.  The row, plane and element strides are read from the header;
the access model is the hardware's: 32 banks of 4 bytes, a warp's scalar accesses in one
wavefront per distinct word and bank, 8-byte accesses per half-warp, 16-byte per quarter-warp."""
import os
import re

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                      "paper_2510_05254_b300", "csrc", "stage_kernel.cuh")


def _header():
    return open(HEADER).read()


def test_strides_are_the_ones_analysed_here():
    h = _header()
    assert re.search(r"RS = VEC \? \(n == 8 \? 12 : 4\) : \(\(DENSE \|\| PLANE\) \? n : n \+ 1\);", h)
    assert re.search(r"PS = PLANE \? n \* n \+ 8 : RS \* n;", h)
    assert re.search(r"SPE = VEC \? \(n == 8 \? 104 : 20\) : \(PLANE \? n \* PS : RS \* L\);", h)
    # line geometry: y-lines step by RS inside a plane, z-lines by PS
    assert "pbase = i + PS * k; pstride = RS;" in h
    assert "pbase = line % n + RS * (line / n); pstride = PS;" in h


def geometry(dim, n, RS, PS, a, line):
    if a == 0:
        return (RS * (line % n) + PS * (line // n) if dim == 3 else RS * line), 1
    if a == 1:
        return line % n + PS * (line // n), RS
    return line % n + RS * (line // n), PS


def wavefronts(words_per_lane, width):
    """words_per_lane: list over the 32 lanes of the first 4-byte word each accesses (width words
    wide).  Returns the wavefronts of the access (the worst group of lanes served together)."""
    group = {1: 32, 2: 16, 4: 8}[width]
    worst = 0
    for g0 in range(0, 32, group):
        banks = {}
        for w0 in words_per_lane[g0:g0 + group]:
            if w0 is None:
                continue
            for w in range(w0, w0 + width):
                banks.setdefault(w % 32, set()).add(w)
        worst = max([worst] + [len(s) for s in banks.values()])
    return worst


def line_access_ways(dim, n, RS, PS, SPE, a, width, nwarps=4):
    L = n ** (dim - 1)
    worst = 0
    for warp in range(nwarps):
        for l in range(0, n, width if a == 0 else 1):
            words = []
            for lane in range(32):
                tid = 32 * warp + lane
                el, line = divmod(tid, L)
                pbase, pstride = geometry(dim, n, RS, PS, a, line)
                words.append(el * SPE + pbase + l * pstride)
            worst = max(worst, wavefronts(words, width if a == 0 else 1))
    return worst


def test_plane_layout_fp32_3d_degree7():
    n, dim = 8, 3
    RS, PS = n, n * n + 8
    SPE = n * PS
    assert SPE == 576 == 9 * 64  # the footprint of the one-slot padding
    assert line_access_ways(dim, n, RS, PS, SPE, 1, 1) == 1  # y-lines conflict-free
    assert line_access_ways(dim, n, RS, PS, SPE, 2, 1) == 1  # z-lines conflict-free
    assert line_access_ways(dim, n, RS, PS, SPE, 0, 4) == 2  # x-lines as float4: 2-way
    # 16-byte alignment of rows and planes (float4 x-lines, 256-byte bulk copies per plane)
    assert (RS * 4) % 16 == 0 and (PS * 4) % 16 == 0 and (SPE * 4) % 16 == 0
    # update quads: eight consecutive quads of a quarter-warp hit distinct 16-byte bank groups
    pad = lambda node: node + (PS - n * n) * (node // (n * n))
    for q0 in range(0, 128, 8):
        assert wavefronts([pad(4 * q) for q in range(q0, q0 + 8)] * 4, 4) == 1


def test_sixteen_byte_layouts_fp32_2d():
    # degree 7: x-lines as float4 and y-lines both conflict-free
    assert line_access_ways(2, 8, 12, 96, 104, 0, 4) == 1
    assert line_access_ways(2, 8, 12, 96, 104, 1, 1) == 1
    # degree 3: y-lines conflict-free, float4 x-lines 2-way -- no element stride gives both (a
    # quarter-warp's two elements need SPE = 16 mod 32 words, the y-lines SPE/4 odd)
    assert line_access_ways(2, 4, 4, 16, 20, 1, 1) == 1
    assert line_access_ways(2, 4, 4, 16, 20, 0, 4) == 2
    both = [spe for spe in range(16, 129, 4)
            if line_access_ways(2, 4, 4, 16, spe, 0, 4) == 1 and line_access_ways(2, 4, 4, 16, spe, 1, 1) == 1]
    assert both == []


def test_unpadded_degree5_layout_fp32_2d():
    n = 6
    dense = dict(RS=n, PS=n * n, SPE=n * n)
    padded = dict(RS=n + 1, PS=(n + 1) * n, SPE=(n + 1) * n)
    assert line_access_ways(2, n, a=0, width=2, **dense) == 1  # x-lines as float2
    assert line_access_ways(2, n, a=1, width=1, **dense) <= line_access_ways(2, n, a=1, width=1, **padded)


E3F_HEADER = os.path.join(os.path.dirname(HEADER), "stage_euler3d_f32.cuh")


def test_element_major_layouts_fp32_3d_euler():
    """euler3d_f32_body keeps each element's four variables together ([element][variable][SPE]);
    the element stride ES sets the banks of a warp whose lines straddle two elements."""
    h = open(E3F_HEADER).read()
    assert "static constexpr int ES = NV * SPE + (PLANE ? 0 : 24);" in h
    assert "static constexpr int PS = PLANE ? n * n + 8 : n * n;" in h
    # degree 5: ES = 4 * 216 + 24 = 888 words (= 24 mod 32, as the variable-major 216)
    n, ES = 6, 4 * 216 + 24
    ways = [line_access_ways(3, n, n, n * n, ES, a, 2 if a == 0 else 1, nwarps=9) for a in range(3)]
    old = [line_access_ways(3, n, n, n * n, 216, a, 2 if a == 0 else 1, nwarps=9) for a in range(3)]
    assert ways == old == [1, 2, 2]
    # the padding that was not chosen: 8 words would make the y-lines 4-way
    assert line_access_ways(3, n, n, n * n, 4 * 216 + 8, 1, 1, nwarps=9) == 4
    # the update's quads: a quarter-warp's eight float4 reads are conflict-free across elements
    for q0 in range(0, 4 * 54, 8):
        words = [divmod(q, 54)[0] * ES + 4 * divmod(q, 54)[1] for q in range(q0, q0 + 8)]
        assert wavefronts(words * 4, 4) == 1
    assert (ES * 4) % 16 == 0 and (216 * 4) % 16 == 0  # bulk-copy destinations 16-byte aligned
    # degree 7: ES = 4 * 576; a warp never leaves its element, so the plane layout's analysis holds
    n, PS = 8, 72
    ES = 4 * n * PS
    assert [line_access_ways(3, n, n, PS, ES, a, 4 if a == 0 else 1, nwarps=8) for a in range(3)] == [2, 1, 1]
