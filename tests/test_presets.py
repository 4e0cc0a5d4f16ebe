"""The named workload presets build and name only real solver options (CPU only)."""
from paper_2210_11797_gb300 import hmg, presets


def test_small_preset_builds():
    workloads, opts = presets.preset("planar16_helmholtz")
    assert len(workloads) == 1 and workloads[0].mesh.ncell == 16 * 16 * 8
    assert opts == {"tol": 1e-10}


def test_every_preset_uses_real_option_names_and_values():
    fields = {name for name, _ in hmg.Options._fields_}
    assert set(presets.OPTIONS) == set(presets.WORKLOADS)
    for name, opts in presets.OPTIONS.items():
        assert set(opts) <= fields, name
        for k, v in opts.items():
            if isinstance(v, str):
                assert v in hmg._NAMED[k], (name, k, v)
