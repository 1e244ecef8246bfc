"""Helpers for the GPU tests: put a workloads.Block on the device and drive
the C ABI through the binding (paper_1303_4538_gb300.sip)."""
import numpy as np

from paper_1303_4538_gb300 import sip


def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return torch


class GpuSystem:
    """One or more blocks on the device with a factored plan."""

    def __init__(self, blocks, alpha=0.92, mode=sip.SIP_MODE_F64, inner=4, x0=None, tile=None,
                 sym_null=False, coef_f32=False, max_spin=0, stall=0, ifaces=None, graphs=0):
        torch = torch_cuda()
        if not isinstance(blocks, (list, tuple)):
            blocks = [blocks]
        self.blocks = blocks
        stream = torch.cuda.current_stream().cuda_stream
        self.ctx = sip.Context(0, stream)
        self.A, self.b, self.x, descs = [], [], [], []
        for n, blk in enumerate(blocks):
            cdt = torch.float32 if coef_f32 else torch.float64
            A = [torch.from_numpy(np.ascontiguousarray(c)).to("cuda", cdt) for c in blk.coef_list()]
            b = torch.from_numpy(blk.b).cuda()
            if x0 is None:
                x = torch.zeros(blk.n, dtype=torch.float64, device="cuda")
            else:
                x = torch.from_numpy(np.ascontiguousarray(x0[n] if isinstance(x0, list) else x0)).cuda()
            coefs = list(A)
            if sym_null:
                coefs[1] = coefs[3] = coefs[5] = None
            descs.append(sip.make_desc(blk.nx, blk.ny, blk.nz, coefs, b, x, symmetric=blk.symmetric,
                                       coef_dtype=1 if coef_f32 else 0))
            self.A.append(A)
            self.b.append(b)
            self.x.append(x)
        opts = sip.default_options(alpha=alpha, mode=mode, inner_iters=inner, max_spin=max_spin,
                                   debug_stall=stall, graphs=graphs)
        if tile:
            opts.tile_j, opts.tile_k = tile[:2]
            if len(tile) > 2:
                opts.rows_per_thread = tile[2]
            if len(tile) > 3:
                opts.stages = tile[3]
        torch.cuda.synchronize()
        ifs = None
        if ifaces:
            ifs = []
            for lo, hi, nj, nk in ifaces:
                f = sip.sip_interface()
                f.blk_lo, f.blk_hi, f.nj, f.nk = lo, hi, nj, nk
                ifs.append(f)
        self.plan = sip.Plan(self.ctx, descs, opts, ifaces=ifs, keep=(self.A, self.b, self.x))

    def xs(self, n=0):
        return self.x[n].cpu().numpy()

    def factors(self, n=0):
        torch = torch_cuda()
        out = [torch.empty(self.blocks[n].n, dtype=torch.float64, device="cuda") for _ in range(7)]
        self.plan.export_factors(n, out)
        return [o.cpu().numpy() for o in out]

    def close(self):
        self.plan.close()
        self.ctx.close()
