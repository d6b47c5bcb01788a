"""Which tcgen05.mma operand kinds the assembler accepts for sm_103a (GB300).

The limb path splits L^{-1} into BF16 integer limbs (kind::f16). An INT8 route
(kind::i8, s8 x s8 -> s32 with exact integer accumulation) would take the int8 dosage
blocks as they arrive, but ptxas refuses that kind for sm_103a while it accepts it for
sm_100a: there is no INT8 tensor rate on this part to build a limb variant on. This test
runs only the assembler (no GPU) on a one-instruction kernel, so the finding is checked
against the installed toolkit every time the CPU suite runs.
"""
import shutil
import subprocess

import pytest

PTXAS = shutil.which("ptxas") or "/usr/local/cuda/bin/ptxas"

KERNEL = """.version 9.0
.target {arch}
.address_size 64
.visible .entry k()
{{
    .reg .b32 r<3>;
    .reg .b64 rd<2>;
    .reg .pred p0;
    mov.b32 r0, 0;
    mov.b32 r1, 0;
    mov.b64 rd0, 0;
    mov.b64 rd1, 0;
    setp.ne.b32 p0, r0, 0;
    tcgen05.mma.cta_group::1.kind::{kind} [r0], rd0, rd1, r1, p0;
    ret;
}}
"""


def assemble(tmp_path, kind, arch):
    src = tmp_path / f"k_{kind}_{arch}.ptx"
    src.write_text(KERNEL.format(kind=kind, arch=arch))
    r = subprocess.run([PTXAS, f"-arch={arch}", str(src), "-o", str(tmp_path / "k.cubin")],
                       capture_output=True, text=True, timeout=120)
    return r.returncode, r.stdout + r.stderr


@pytest.fixture(scope="module")
def have_ptxas():
    if not (shutil.which("ptxas") or shutil.which(PTXAS)):
        pytest.skip("ptxas not installed")


@pytest.mark.parametrize("arch", ["sm_100a", "sm_103a"])
def test_kind_f16_assembles(tmp_path, have_ptxas, arch):
    rc, out = assemble(tmp_path, "f16", arch)
    assert rc == 0, out


def test_kind_i8_exists_for_sm100a_only(tmp_path, have_ptxas):
    rc, out = assemble(tmp_path, "i8", "sm_100a")
    assert rc == 0, out
    rc, out = assemble(tmp_path, "i8", "sm_103a")
    assert rc != 0
    assert "kind::i8" in out and "not supported" in out, out
