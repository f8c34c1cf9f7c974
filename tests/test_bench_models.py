"""Every kernel span the library can trace has an entry in the bench's roofline
model (CPU only: a check of the sources)."""
import re
from pathlib import Path

ROOT = Path(__file__).resolve().parents[1]


def _traced_names():
    names = set()
    for f in (ROOT / "paper_1504_04653_gb300" / "csrc").glob("*.cu"):
        for call in re.findall(r"trace_mark\(pl, \w+, ([^;]*)\);", f.read_text()):
            names.update(re.findall(r'"(k_\w+)"', call))
    return names


def test_every_traced_kernel_is_modelled():
    names = _traced_names()
    assert {"k_table", "k_sample_pband", "k_f32_split_w8", "k_f64_band_pass", "k_df_band_pass"} <= names
    src = (ROOT / "bench.py").read_text()
    body = src[src.index("def kernel_models("):src.index("def roofline(")]
    missing = sorted(n for n in names if f'"{n}"' not in body and n not in ("k_convolve", "k_apply",
                                                                               "k_sample_coupling", "k_sample_tiles"))
    assert not missing, missing
    # the kernels outside the step get their models where the bench times them
    for n in ("k_convolve", "k_apply", "k_sample_coupling", "k_sample_tiles"):
        assert f'roofline("{n}"' in src, n
