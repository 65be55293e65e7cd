"""The TMA tile-load plan (rt_tma_plan, host logic in csrc/rt_tma_plan.h, no
device needed): which device instances the tile kernels fetch with tensor
copies. Groups are maximal runs of consecutive instances of one shape with
16-byte rows and room for every tile box (nx >= 72, ny >= 36), at most 4,
largest first (cells times instances), ties to the earlier run."""
import pytest


def _rt():
    import paper_2608_04085_b300 as rt
    return rt


def test_uniform_batch_is_one_group():
    g, k = _rt().tma_plan([(256, 768)] * 32)
    assert g == [0] * 32 and k == list(range(32))


def test_uneven_batch_groups_largest_first():
    shapes = [(128, 384)] * 32 + [(256, 768)] * 24 + [(512, 1536)] * 8
    g, k = _rt().tma_plan(shapes)
    # cells x instances: 8 x 512 x 1536 > 24 x 256 x 768 > 32 x 128 x 384
    assert g == [2] * 32 + [1] * 24 + [0] * 8
    assert k == list(range(32)) + list(range(24)) + list(range(8))


def test_row_alignment_and_minimum_sizes():
    rt = _rt()
    # 98 columns: 392-byte FP32 rows are not a multiple of 16 bytes, 784-byte FP64 rows are
    assert rt.tma_plan([(98, 90)], 4)[0] == [-1]
    assert rt.tma_plan([(98, 90)], 8)[0] == [0]
    assert rt.tma_plan([(100, 90)], 4)[0] == [0]
    # too narrow for a box plus a tile, too short for the tallest box
    assert rt.tma_plan([(64, 192), (72, 36), (128, 35)], 4)[0] == [-1, 0, -1]


def test_runs_are_consecutive_and_at_most_four_are_kept():
    rt = _rt()
    A, B = (128, 96), (96, 72)
    # equal shapes that are not neighbours form separate runs (separate tensors)
    g, k = rt.tma_plan([A, B, A], 4)
    assert g == [0, 2, 1] and k == [0, 0, 0]
    # six runs: the two smallest (by cells x instances) keep plain loads; the
    # tie between the two equal A runs goes to the earlier one
    shapes = [A, A, B, (160, 64), A, A, (72, 40), (104, 80)]
    g, _ = rt.tma_plan(shapes, 4)
    # run sizes: A,A 24576; B 6912; 160x64 10240; A,A 24576; 72x40 2880; 104x80 8320
    assert g == [0, 0, -1, 2, 1, 1, -1, 3]


def test_bad_arguments():
    rt = _rt()
    with pytest.raises(rt.RtError):
        rt.tma_plan([(256, 768)], 2)
    assert rt.tma_plan([], 4) == ([], [])
