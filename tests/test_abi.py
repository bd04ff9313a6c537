"""Host-side checks of the C ABI: the library loads without a GPU, exports every
function include/nlse.h declares, and validates arguments before any CUDA call."""
import ctypes
import os
import re

import pytest

from paper_2306_15678_gb300 import capi, configs
from paper_2306_15678_gb300.grid import make_params

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"^\s*(?:const\s+)?\w+\*?\s+\*?(nlse_\w+)\s*\(", txt, re.M))
    return sorted(names)


def test_library_exports_every_declared_function():
    lib = capi.lib()
    decl = declared_functions()
    assert len(decl) >= 14
    for name in decl:
        assert hasattr(lib, name), name
    assert set(decl) == set(capi.exported_symbols())


def test_status_strings_and_version():
    for s in range(8):
        assert capi.nlse_status_string(s).startswith("NLSE")
    assert capi.nlse_version() >= 10000


def test_workspace_size_and_validation_on_host():
    cfg = configs.cfg_dense_fp32()
    p = make_params(cfg)
    ws = capi.nlse_workspace_size(p)
    assert ws >= 2 * 4096 * 4096 * 8
    p64 = make_params(cfg, precision="fp64")
    assert capi.nlse_workspace_size(p64) >= 2 * 4096 * 4096 * 16
    bad = [("n", 100, capi.NLSE_EINVAL), ("n", 16384, capi.NLSE_EUNSUPPORTED),
           ("n", 4, capi.NLSE_EUNSUPPORTED), ("precision", 7, capi.NLSE_EUNSUPPORTED),
           ("K", 0, capi.NLSE_EINVAL), ("terms", 16, capi.NLSE_EINVAL),
           ("L", -1.0, capi.NLSE_EINVAL), ("dz", 0.0, capi.NLSE_EINVAL),
           ("diag_every", -1, capi.NLSE_EINVAL), ("scheme", 4, capi.NLSE_EINVAL)]
    for field, val, code in bad:
        q = make_params(cfg)
        setattr(q, field, val)
        with pytest.raises(capi.NlseError) as ei:
            capi.nlse_workspace_size(q)
        assert ei.value.status == code, (field, val)


def test_create_rejects_bad_workspace_before_any_launch():
    p = make_params(configs.cfg_plain_fp64())
    with pytest.raises(capi.NlseError) as ei:
        capi.nlse_create(p, 0, 0, 1 << 20)
    assert ei.value.status == capi.NLSE_EINVAL
    with pytest.raises(capi.NlseError) as ei:
        capi.nlse_create(p, 0, 256 * 1024, 1024)  # too small: ENOMEM before touching it
    assert ei.value.status == capi.NLSE_ENOMEM
    with pytest.raises(capi.NlseError) as ei:
        capi.nlse_create(p, 0, 256 * 1024 + 8, 1 << 40)  # misaligned
    assert ei.value.status == capi.NLSE_EINVAL


def test_large_adjoint_fits_with_sqrt_checkpointing():
    """8192^2 FP32, 3000 steps (the large batched adjoint): checkpointing every
    ceil(sqrt(3000)) = 55 steps keeps one beam's workspace near 2 sqrt(M) fields
    (~56 GiB), so several beams fit in the GPU's memory at once; storing every
    step would need 3000 fields (1.5 TiB)."""
    cfg = configs.cfg_large_adjoint(1)[0]
    p = make_params(cfg)
    M = cfg["nsteps"]
    k = configs.sqrt_checkpoint(M)
    assert k == 55
    field = 8192 * 8192 * 8
    ws = capi.nlse_adjoint_workspace_size(p, M, k)
    nck = -(-M // k)
    assert (k + nck) * field <= ws <= (k + nck + 6) * field
    assert ws < 60 * 2 ** 30
    assert capi.nlse_adjoint_workspace_size(p, M, M) > 25 * ws


def test_symmetric_steps_only_for_single_grids():
    """The batched march and the adjoint take Lie steps only: asking either for
    the symmetric scheme is NLSE_EUNSUPPORTED, on the host, before any launch."""
    cfg = dict(configs.scaled(configs.cfg_dense_fp32(), 512), scheme="strang")
    p = make_params(cfg)
    assert p.scheme == capi.NLSE_STRANG
    assert capi.nlse_workspace_size(p) > 0
    with pytest.raises(capi.NlseError) as ei:
        capi.nlse_adjoint_workspace_size(p, 10, 5)
    assert ei.value.status == capi.NLSE_EUNSUPPORTED
    with pytest.raises(capi.NlseError) as ei:
        capi.nlse_batch_workspace_size([p])
    assert ei.value.status == capi.NLSE_EUNSUPPORTED
    with pytest.raises(ValueError):
        make_params(dict(cfg, scheme="leapfrog"))


def test_lens_scratch_size_and_null_checks():
    """The effective lens's scratch: counters, a complex work array, labels,
    64-bit keys and centres per point; host-only, validates the parameters."""
    cfg = configs.cfg_dense_fp32()
    p = make_params(cfg)
    n = p.n
    assert capi.nlse_lens_scratch_size(p) >= n * n * (8 + 4 + 8 + 4)
    p64 = make_params(cfg, precision="fp64")
    assert capi.nlse_lens_scratch_size(p64) >= n * n * (16 + 4 + 8 + 4)
    q = make_params(cfg)
    q.n = 100
    with pytest.raises(capi.NlseError) as ei:
        capi.nlse_lens_scratch_size(q)
    assert ei.value.status == capi.NLSE_EINVAL
    lens = capi.make_lens(dict(l_dif=1e-4, w_l=1e11, re=[(0.1, 1.0, 1.0, 0.0)]))
    with pytest.raises(capi.NlseError) as ei:
        capi.nlse_effective_lens(None, lens, 0, 0, 0, 0, 0)
    assert ei.value.status == capi.NLSE_EINVAL
    with pytest.raises(ValueError):
        capi.make_lens(dict(l_dif=0.0, w_l=1.0, re=[(0.1 * (j + 1), 1, 1, 0) for j in range(9)]))


def test_exact_screen_validation_on_host():
    """The exact substep takes real gains and K >= 2; the batched march and the
    adjoint take the plain Lie step only."""
    cfg = dict(configs.cfg_plain_fp64(), screen="exact")
    p = make_params(cfg)
    assert p.scheme == capi.NLSE_EXACT_SCREEN
    assert capi.nlse_workspace_size(p) > 0
    p.scheme = capi.NLSE_STRANG | capi.NLSE_EXACT_SCREEN
    assert capi.nlse_workspace_size(p) > 0
    for field, val in (("theta", (1.0, 0.1, 1.0, 0.0, 1.0, 0.0)), ("K", 1)):
        q = make_params(cfg)
        if field == "theta":
            for i, t in enumerate(val):
                q.theta[i] = t
        else:
            q.K = val
        with pytest.raises(capi.NlseError) as ei:
            capi.nlse_workspace_size(q)
        assert ei.value.status == capi.NLSE_EINVAL
    q = make_params(cfg)
    q.scheme = 4
    with pytest.raises(capi.NlseError) as ei:
        capi.nlse_workspace_size(q)
    assert ei.value.status == capi.NLSE_EINVAL
    with pytest.raises(capi.NlseError) as ei:
        capi.nlse_adjoint_workspace_size(make_params(cfg), 10, 2)
    assert ei.value.status == capi.NLSE_EUNSUPPORTED
    with pytest.raises(ValueError):
        make_params(dict(cfg, screen="implicit"))


def test_ctypes_records_match_the_c_header_layout(tmp_path):
    """Field offsets and sizes of the ctypes mirrors (nlse_params,
    nlse_batch_tuning, nlse_lens) equal those gcc computes from
    include/nlse.h, so every field the binding sets lands where the library
    reads it."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    records = {"nlse_params": capi.nlse_params, "nlse_batch_tuning": capi.nlse_batch_tuning,
               "nlse_lens": capi.nlse_lens}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "nlse.h"', "int main(void) {"]
    for name, cls in records.items():
        lines.append(f'printf("{name} sizeof %zu\\n", sizeof({name}));')
        for fname, _ in cls._fields_:
            lines.append(f'printf("{name} {fname} %zu\\n", offsetof({name}, {fname}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run([gcc, "-std=c11", "-I", inc, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for line in out:
        if line.strip():
            rec, field, val = line.split()
            got[(rec, field)] = int(val)
    for name, cls in records.items():
        assert got[(name, "sizeof")] == ctypes.sizeof(cls), name
        for fname, _ in cls._fields_:
            assert got[(name, fname)] == getattr(cls, fname).offset, (name, fname)


def test_batch_workspace_size_and_validation_on_host():
    """Batch sizing needs no GPU: the workspace grows with the beams' fields and
    their 256 dithered table copies, and sizes or precisions the batched
    kernel does not take are refused before any CUDA call."""
    base = configs.cfg_dense_fp32()
    p512 = make_params(configs.scaled(base, 512), "fp32")
    p2048 = make_params(configs.scaled(base, 2048), "fp32")
    one = capi.nlse_batch_workspace_size([p512])
    two = capi.nlse_batch_workspace_size([p512, p512])
    mixed = capi.nlse_batch_workspace_size([p512, p2048])
    assert one >= 512 * 512 * 8 and two > one and mixed > two
    # the second 512^2 beam adds its field and propagator copies, not another twiddle block
    assert two - one < 512 * 512 * 8 + 256 * (512 * 8 + 24 * 256) + 4096
    for bad, status in ((make_params(configs.scaled(base, 128), "fp32"), capi.NLSE_EUNSUPPORTED),
                        (make_params(configs.scaled(base, 512), "fp64"), capi.NLSE_EUNSUPPORTED)):
        with pytest.raises(capi.NlseError) as ei:
            capi.nlse_batch_workspace_size([bad])
        assert ei.value.status == status
