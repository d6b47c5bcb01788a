"""gwas_stream, the native out-of-core driver: files in (relatedness, covariates,
phenotypes; int8 dosages or a SNP-major PLINK .bed), block-streamed through the C ABI
with the file reads overlapped, files out; results against the oracle."""
import json
import subprocess

import numpy as np
import pytest

import synth
from oracle import gls as G


def cli():
    from paper_1304_2272_gb300 import build
    build.build()
    return str(build.CLI)


def write_inputs(tmp, c, X):
    np.ascontiguousarray(c.phi).tofile(tmp / "phi.f64")     # symmetric: either order
    np.ascontiguousarray(c.XL.T).tofile(tmp / "covar.f64")  # column-major n x q
    np.ascontiguousarray(c.Y.T).tofile(tmp / "pheno.f64")
    np.ascontiguousarray(X.T).tofile(tmp / "dos.i8")        # one SNP after another
    P = synth.pack_2bit(X, call_of=(3, 2, 0), missing_call=1)   # PLINK: 00 = two copies
    with open(tmp / "g.bed", "wb") as f:
        f.write(bytes([0x6C, 0x1B, 0x01]))
        f.write(np.ascontiguousarray(P.T).tobytes())


def run_cli(args):
    return subprocess.run([cli(), *map(str, args)], capture_output=True, text=True, timeout=600)


def test_usage_and_bad_inputs(tmp_path):
    assert run_cli([]).returncode == 1
    (tmp_path / "bad.bed").write_bytes(b"\x00\x01\x02" + bytes(100))
    for f in ("phi.f64", "covar.f64", "pheno.f64"):
        (tmp_path / f).write_bytes(bytes(8))
    r = run_cli(["--n", 4, "--q", 1, "--phi", tmp_path / "phi.f64", "--covar",
                 tmp_path / "covar.f64", "--pheno", tmp_path / "pheno.f64", "--bed",
                 tmp_path / "bad.bed", "--m", 3, "--out", tmp_path / "o"])
    assert r.returncode == 3 and "PLINK" in r.stderr


@pytest.mark.gpu
@pytest.mark.parametrize("fmt,precision,tol", [("int8", "fp64", 1e-10), ("bed", "fp64", 1e-10),
                                               ("bed", "mixed", 1e-6)])
def test_stream_matches_oracle(gpu, tmp_path, fmt, precision, tol):
    n, m, t = 301, 1000, 2
    c = synth.make_cohort(71, n, t=t, n_markers=300)
    X = c.snps(m).copy(order="F")
    X[3, 10] = -1          # missing / bad call
    X[:, 20] = 1           # constant: singular with the intercept
    write_inputs(tmp_path, c, X)
    src = ["--dosages", tmp_path / "dos.i8"] if fmt == "int8" else ["--bed", tmp_path / "g.bed"]
    r = run_cli(["--n", n, "--q", 3, "--t", t, "--phi", tmp_path / "phi.f64", "--covar",
                 tmp_path / "covar.f64", "--pheno", tmp_path / "pheno.f64", *src, "--m", m,
                 "--m-blk", 256, "--h", c.h, "--sigma2", c.sigma2, "--precision", precision,
                 "--out", tmp_path / "o"])
    assert r.returncode == 0, r.stderr
    info = json.loads(r.stdout.strip().splitlines()[-1])
    assert info["m"] == m and info["input"] == fmt
    b = np.fromfile(tmp_path / "o.b", dtype=np.float64).reshape(m, t, 4)
    st = np.fromfile(tmp_path / "o.status", dtype=np.uint8)
    rb, rw, rs = G.gls(c.phi, c.h, c.sigma2, c.XL, c.Y, X)
    np.testing.assert_array_equal(st, rs)
    assert st[10] == 2 and st[20] == 1 and info["status_ok"] == int((rs == 0).sum())
    ok = rs == 0
    scale = np.max(np.abs(rb[ok]), axis=-1, keepdims=True)
    assert np.max(np.abs(b[ok] - rb[ok]) / scale) <= tol


@pytest.mark.gpu
def test_short_genotype_file_is_an_error(gpu, tmp_path):
    c = synth.make_cohort(72, 100, n_markers=100)
    X = c.snps(50)
    write_inputs(tmp_path, c, X)
    r = run_cli(["--n", 100, "--q", 3, "--phi", tmp_path / "phi.f64", "--covar",
                 tmp_path / "covar.f64", "--pheno", tmp_path / "pheno.f64", "--dosages",
                 tmp_path / "dos.i8", "--m", 80, "--m-blk", 32, "--out", tmp_path / "o"])
    assert r.returncode == 4 and "short read" in r.stderr


@pytest.mark.gpu
def test_checkpoint_and_resume(gpu, tmp_path):
    """A job stopped after 2 of its 5 blocks and resumed writes the same bytes as one
    uninterrupted run; a resume with other job sizes is refused."""
    n, m = 257, 300
    c = synth.make_cohort(73, n, n_markers=300)
    X = c.snps(m)
    write_inputs(tmp_path, c, X)
    base = ["--n", n, "--q", 3, "--phi", tmp_path / "phi.f64", "--covar", tmp_path / "covar.f64",
            "--pheno", tmp_path / "pheno.f64", "--bed", tmp_path / "g.bed", "--m", m,
            "--m-blk", 64, "--h", c.h, "--sigma2", c.sigma2]
    full = run_cli([*base, "--out", tmp_path / "full"])
    assert full.returncode == 0, full.stderr
    first = run_cli([*base, "--checkpoint", "--max-blocks", 2, "--out", tmp_path / "part"])
    assert first.returncode == 0, first.stderr
    info = json.loads(first.stdout.strip().splitlines()[-1])
    assert info["blocks_done"] == 2 and info["blocks"] == 5 and info["complete"] is False
    assert (tmp_path / "part.progress").read_text().strip().endswith("blocks=2")
    rest = run_cli([*base, "--resume", "--out", tmp_path / "part"])
    assert rest.returncode == 0, rest.stderr
    info = json.loads(rest.stdout.strip().splitlines()[-1])
    assert info["first_block"] == 2 and info["complete"] is True
    for ext in (".b", ".wald", ".status"):
        assert (tmp_path / ("part" + ext)).read_bytes() == (tmp_path / ("full" + ext)).read_bytes()
    other = [*base[:-6], "--m-blk", 32, "--h", c.h, "--sigma2", c.sigma2]
    bad = run_cli([*other, "--resume", "--out", tmp_path / "part"])
    assert bad.returncode == 6 and "another job" in bad.stderr
    # another model (h) or other phenotype values on the same sizes are another job too
    first = run_cli([*base, "--checkpoint", "--max-blocks", 2, "--out", tmp_path / "p2"])
    assert first.returncode == 0, first.stderr
    other_h = [*base[:-4], "--h", c.h + 0.1, "--sigma2", c.sigma2]
    bad = run_cli([*other_h, "--resume", "--out", tmp_path / "p2"])
    assert bad.returncode == 6 and "another job" in bad.stderr
    np.ascontiguousarray(c.Y.T + 1.0).tofile(tmp_path / "pheno.f64")
    bad = run_cli([*base, "--resume", "--out", tmp_path / "p2"])
    assert bad.returncode == 6 and "another job" in bad.stderr
