"""Host-side scheduling of the split GEMM (no GPU needed): ccsd_split_describe reports how
ccsd_split_zgemm would run a shape (kernel, orientation, tile width, cluster, K split, tiles).

Without a GPU the cluster occupancy query fails and every launch plans one CTA per tile
(cluster 1); on a GB300 the outputs two or four tiles wide take clusters of two. Both are
accepted below; the orientation, tile width and tile counts do not depend on the device.
"""
import pytest

from paper_2103_08473_gb300 import build, ccsd


@pytest.fixture(scope="module")
def lib():
    return ccsd.load(build.build())


def test_ladder_shape_swaps_the_short_pair_side_onto_two_96_wide_tiles(lib):
    # o20/v120 ladder: tau's 190 pair rows against 7140 pair rows of <ab||cd>, K = 7140
    d = ccsd.split_describe(190, 7140, 7140)
    assert d["short_k"] == 0 and d["swap"] == 1 and d["tile_n"] == 96
    assert d["tiles"] == 56 * 2  # 7140 rows on the 128-row side, 190 on two 96-wide tiles
    assert d["cluster"] in (1, 2)
    assert d["ksplits"] >= 2  # 112 tiles are fewer than the SMs: K is split to fill them


def test_short_k_products_take_the_short_k_kernel(lib):
    # t1 (20 rows) times the unpacked <ak||cd> rows over K = v = 120: one K block
    assert ccsd.split_describe(20, 288000, 120)["short_k"] == 1
    # four blocks of 128 e4m3 digits are the limit
    assert ccsd.split_describe(256, 256, 512)["short_k"] == 1
    assert ccsd.split_describe(256, 256, 513)["short_k"] == 0


def test_square_product_keeps_the_plain_orientation(lib):
    d = ccsd.split_describe(2400, 2400, 2400)  # the (ov)^3 products at o20/v120
    assert d == {"short_k": 0, "swap": 0, "tile_n": 128, "cluster": 1, "ksplits": 1, "tiles": 19 * 19}


def test_two_and_four_tile_outputs_may_pair_into_clusters(lib):
    for M, N, tiles in [(2000, 200, 16 * 2), (1000, 500, 8 * 4)]:
        d = ccsd.split_describe(M, N, 1500)
        assert d["short_k"] == 0 and d["swap"] == 0 and d["tile_n"] == 128 and d["tiles"] == tiles
        assert d["cluster"] in (1, 2)


def test_describe_rejects_bad_configurations(lib):
    for args in [(10, 10, 10, 0, 6, 8), (10, 10, 10, 0, 5, 0), (-1, 10, 10, 0, 5, 8), (10, 10, 10, 7, 5, 8)]:
        M, N, K, kind, bits, slices = args
        with pytest.raises(ccsd.CCSDError):
            ccsd.split_describe(M, N, K, kind=kind, bits=bits, slices=slices)


def test_skinny_long_k_products_split_k_across_the_gpu(lib):
    # H^k_i at o20/v120: a 20 x 20 output over K = 288000 (2250 blocks of 128 digits). One output
    # tile: K is split so that the CTAs cover the GPU, each split keeping >= 6 K blocks.
    d = ccsd.split_describe(20, 20, 288000)
    assert d["short_k"] == 0 and d["tiles"] == 1
    assert 100 <= d["ksplits"] <= 2250 // 6
