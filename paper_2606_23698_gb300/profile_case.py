"""One small, self-contained GPU invocation for profiler captures.

    python -m paper_2606_23698_gb300.profile_case stage D0 D1 D2 AXIS STAGE MODE
    python -m paper_2606_23698_gb300.profile_case fft3 D0 D1 D2 MODE
    python -m paper_2606_23698_gb300.profile_case ablation

`stage` runs a single stage launch (Bailey stage 1 or 2 of one axis pass) of a
D0 x D1 x D2 plan on seeded uniform input; `fft3` runs one forward transform;
`ablation` runs each epilogue ablation kernel once (4 Phase-B word layouts,
3 residue forms; 2^22 items from 2^16 L2-resident inputs, 16 perturbed
repetitions each).
Both print one line and exit 0, so the same command can run once plainly and
then under a profiler restricted to the kernel of interest.
"""
import sys

import torch

from synth import inputs as S

from .api import Plan


def main(argv):
    what = argv[0]
    shape = tuple(int(v) for v in argv[1:4]) if what != "ablation" else None
    if what == "stage":
        axis, stage, mode = int(argv[4]), int(argv[5]), argv[6]
        pl = Plan(*shape, mode=mode)
        x = S.complex_uniform(1, shape, device="cuda").to(pl.dtype)
        out = torch.empty_like(x)
        pl.exec_stage(axis, stage, x, out)
    elif what == "fft3":
        mode = argv[4]
        pl = Plan(*shape, mode=mode)
        x = S.complex_uniform(1, shape, device="cuda").to(pl.dtype)
        out = torch.empty_like(x)
        pl.exec(x, out)
    elif what == "ablation":
        from . import _lib
        from .ablation import PHASE_B_VARIANTS, RESIDUE_VARIANTS, phase_b_inputs, residue_inputs
        import numpy as np
        nu, nt = 1 << 16, 1 << 22
        acc, et = phase_b_inputs(nu)
        dacc, det = torch.from_numpy(acc.view(np.int32)).cuda(), torch.from_numpy(et).cuda()
        ck = torch.zeros(1, dtype=torch.int64, device="cuda")
        for v in PHASE_B_VARIANTS:
            _lib.obfft_ablation_phase_b(v, nu, nt, dacc.data_ptr(), det.data_ptr(), None, ck.data_ptr(), reps=16)
        xt = torch.from_numpy(residue_inputs(nu)).cuda()
        for v in RESIDUE_VARIANTS:
            _lib.obfft_ablation_residues(v, nu, nt, xt.data_ptr(), None, ck.data_ptr(), reps=16)
        torch.cuda.synchronize()
        print("ok ablation", int(ck.item()))
        return
    else:
        raise SystemExit(f"unknown case {what!r}")
    torch.cuda.synchronize()
    print("ok", what, shape, float(out.abs().sum()))


if __name__ == "__main__":
    main(sys.argv[1:])
