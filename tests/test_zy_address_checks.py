"""The address-checked debug build (libmpdo_bounds.so: the same sources compiled with -DMPDO_BOUNDS).

Its kernels check every global-memory access against the live device ranges (the library's own
allocations and the buffers a caller registers) and, instead of touching memory outside them, count
the access and record the first one (no trap, no fault).  Two things are tested:
1. A selection of the GPU tests (every update route, precision mode, readout, the batched runtime,
   graphs, the tensor-core GEMM and the failure paths) runs again under the checked library, in a
   child process (the binding chooses its library when it loads); the conftest fixture fails every
   test after which a check failed, so the selection passes only with no out-of-range access.
2. A failed check is reported: a batched gate whose channel-index array was never registered (valid
   memory, so nothing can fault either way) is recorded at the gate-fusion kernel, and once the
   array is registered the same call runs clean and matches the oracle.
The file sorts after the other GPU tests so that they run first under -x."""
import json
import os
import subprocess
import sys

import pytest

from paper_2508_07610_gb300 import build as B

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SELECTION = " or ".join([
    "smallest_caps", "three_qubit_channels_match", "global_bond_truncation_matches", "kraus_first_order",
    "batch_with_per_chain", "batch_channel_index", "graph_capture", "checkpoint",
    "neighbour_truncation_matches", "tiny_norm", "batched_global_bond", "distribution_matches",
    "tc_gemm_matches", "non_finite", "bounded_wait", "trace_guard",
])
FILES = ["tests/test_gpu_parity.py", "tests/test_gpu_batched.py", "tests/test_gpu_analysis.py",
         "tests/test_gpu_tensor_cores.py", "tests/test_gpu_failures.py"]


@pytest.fixture(scope="module")
def checked_env():
    B.build(bounds=True)
    env = dict(os.environ)
    env["MPDO_LIBRARY"] = "bounds"
    env["PYTHONPATH"] = ROOT + (os.pathsep + env["PYTHONPATH"] if env.get("PYTHONPATH") else "")
    return env


def test_gpu_tests_run_clean_under_address_checks(checked_env):
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu", "-p", "no:cacheprovider",
                        *FILES, "-k", SELECTION], cwd=ROOT, env=checked_env, capture_output=True, text=True,
                       timeout=1800)
    tail = r.stdout[-4000:] + "\n" + r.stderr[-2000:]
    print(tail)
    assert r.returncode == 0, tail
    summary = [s for s in r.stdout.splitlines() if " passed" in s][-1]
    assert "failed" not in summary and "error" not in summary, summary


DETECT = r"""
import json
import numpy as np
import torch
from oracle import channels as OC
from oracle import mpdo as OM
from paper_2508_07610_gb300 import mpdo as G
from paper_2508_07610_gb300 import workloads as W

assert G.bounds_enabled()
out = {"before": G.bounds_read()["failures"]}
rng = np.random.default_rng(3)
chi = W.kraus_to_chi(W.random_channel_kraus(2, 3, rng))
U = W.random_unitary(4, rng)
B = 2
U_dev = torch.tensor(np.stack([U] * B), dtype=torch.complex128, device="cuda")
idx_dev = torch.zeros(B, dtype=torch.int32, device="cuda")
G.bounds_register(U_dev.data_ptr(), U_dev.numel() * U_dev.element_size())
stream = torch.cuda.current_stream().cuda_stream
for registered in (False, True):
    if registered:
        G.bounds_register(idx_dev.data_ptr(), idx_dev.numel() * idx_dev.element_size())
    st = G.MPDO(3, 4, 2, "fp64", batch=B, stream=stream)
    cs = st.channels(2, [chi])
    st.apply_2q_batch(0, U_dev.data_ptr(), cs, idx_dev.data_ptr())
    st.sync()
    rep = G.bounds_read()
    o = OM.MPDO(3, 4, 2)
    o.apply_2q(0, U, OC.chi_to_kraus(chi, 2))
    rho = st.sites(1)
    g = OM.MPDO(3, 4, 2)
    g.sites = rho
    err = float(np.max(np.abs(g.dense() - o.dense())))
    out["registered" if registered else "unregistered"] = {"report": rep, "err": err}
print("RESULT " + json.dumps(out))
"""


def test_unregistered_buffer_is_reported(checked_env):
    r = subprocess.run([sys.executable, "-c", DETECT], cwd=ROOT, env=checked_env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-3000:]
    line = [s for s in r.stdout.splitlines() if s.startswith("RESULT ")][-1]
    out = json.loads(line[len("RESULT "):])
    print(out)
    assert out["before"] == 0
    bad, good = out["unregistered"], out["registered"]
    # every chain's channel index is read once by the fusion kernel: B failed checks, the first at
    # its source line, 4 bytes wide, inside the unregistered array
    assert bad["report"]["failures"] >= 1
    assert bad["report"]["file"] == "mpdo_kernels.cu" and bad["report"]["line"] > 0
    assert bad["report"]["bytes"] == 4
    assert good["report"]["failures"] == 0
    assert good["err"] < 1e-12
