"""Host-side checks of the C-ABI library: it builds, loads, and exports every
symbol include/mppi.h declares; the ctypes config mirrors the C struct.  No
compute calls (these run without a GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mppi.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mppi_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def built():
    from paper_2603_07199_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("mppi_create", "mppi_set_gates", "mppi_set_sdf_weights", "mppi_step", "mppi_get_nominal",
              "mppi_destroy", "mppi_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(built):
    lib = ctypes.CDLL(built)
    for name in _declared():
        assert hasattr(lib, name), name
    from paper_2603_07199_gb300 import binding
    assert sorted(binding.EXPORTS) == _declared()


def test_config_struct_layout_matches_header(built, tmp_path):
    src = tmp_path / "sz.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "mppi.h"\n'
                   'int main(void){printf("%zu %zu %zu\\n", sizeof(mppi_config), offsetof(mppi_config, seed),'
                   ' offsetof(mppi_config, softplus_beta)); return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    size, off_seed, off_beta = map(int, subprocess.run([str(exe)], capture_output=True, text=True,
                                                       check=True).stdout.split())
    from paper_2603_07199_gb300 import binding
    assert ctypes.sizeof(binding.MppiConfig) == size
    assert binding.MppiConfig.seed.offset == off_seed
    assert binding.MppiConfig.softplus_beta.offset == off_beta


def test_defaults_and_create_without_gpu(built):
    from paper_2603_07199_gb300 import binding
    cfg = binding.mppi_config_default()
    assert (cfg.K, cfg.H, cfg.max_gates) == (256, 20, 1)
    assert abs(cfg.lam - 0.1) < 1e-7 and abs(cfg.softplus_beta - 100.0) < 1e-5
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:
        has_gpu = False
    if not has_gpu:
        with pytest.raises(binding.MppiError) as e:
            binding.mppi_create(cfg)
        assert e.value.code == binding.MPPI_E_UNSUPPORTED


def test_server_and_other_struct_layouts_match_header(built, tmp_path):
    """Every struct the binding mirrors has the header's size (a field added on one side only
    would shift the others')."""
    src = tmp_path / "sz2.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "mppi.h"\n'
                   'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu\\n", sizeof(mppi_server_config),'
                   ' offsetof(mppi_server_config, batching), offsetof(mppi_server_config, sdf_single_cta),'
                   ' sizeof(mppi_server_stats),'
                   ' offsetof(mppi_server_stats, batches), sizeof(mppi_train_config), sizeof(mppi_depth_camera));'
                   ' return 0;}\n')
    exe = tmp_path / "sz2"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    vals = list(map(int, subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()))
    from paper_2603_07199_gb300 import binding
    assert vals == [ctypes.sizeof(binding.MppiServerConfig), binding.MppiServerConfig.batching.offset,
                    binding.MppiServerConfig.sdf_single_cta.offset, ctypes.sizeof(binding.MppiServerStats), binding.MppiServerStats.batches.offset,
                    ctypes.sizeof(binding.MppiTrainConfig), ctypes.sizeof(binding.MppiDepthCamera)]


def test_server_config_defaults_and_validation_without_gpu(built):
    """The server's defaults (FP16, batched, 16 in flight, single-CTA SDF kernels) and the
    rejection of an out-of-range kernel-form flag, which happens before any device call."""
    from paper_2603_07199_gb300 import binding
    cfg = binding.mppi_server_config_default()
    assert (cfg.sdf_mode, cfg.batching, cfg.max_inflight, cfg.sdf_single_cta, cfg.hbm_budget_bytes) == \
        (binding.MPPI_SDF_MLP_FP16, 1, 16, 1, 0)
    for bad in (-1, 2):
        cfg.sdf_single_cta = bad
        with pytest.raises(binding.MppiError) as e:
            binding.mppi_server_create(cfg)
        assert e.value.code == binding.MPPI_E_INVALID
        assert "sdf_single_cta" in str(e.value)
