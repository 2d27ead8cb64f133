"""The benchmark's description of the fused-sweep variants stays in step with
the library's encoding (include/fm.h, fm_tuning): every variant has a kernel
name for the single solver and the batch, and the sweeps one launch runs
(which turn launch times into per-sweep rooflines) agree with that name.
No GPU needed."""
import bench
from paper_1503_07416_gb300 import fm


def test_every_variant_has_a_kernel_and_a_sweep_count():
    for v in range(fm.FM_SWEEP_VARIANTS):
        spl = bench.sweeps_per_launch(v)
        assert spl in (1, 2), v
        single = bench.sweep_kernel(v, False)
        batched = bench.sweep_kernel(v, True)
        assert single.startswith("k_") and batched.startswith("kb_"), v
        two = "two sweeps" in single or "passes in one cooperative launch" in single
        assert two == (spl == 2), (v, single)
        # the batch runs every variant as one of its own kernels with the same sweep count
        assert ("two sweeps" in batched) == (spl == 2), (v, batched)


def test_tile_shapes_named_for_the_small_and_balanced_tiles():
    assert "16x16" in bench.sweep_kernel(30, False) and "16x8" in bench.sweep_kernel(33, False)
    assert "32x14" in bench.sweep_kernel(35, False)
    assert bench.sweeps_per_launch(35) == 2 and bench.sweeps_per_launch(28) == 1
