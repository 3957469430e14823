"""Test helpers around the C ABI: run the library on a problem and read its
sketches / cores back in the oracle's dict-of-arrays form."""
import numpy as np

from paper_2412_06111_gb300 import api


class Run:
    """A plan + state on the GPU for one (tree, dims, ranks, oversample, seed)."""

    def __init__(self, tree, dims, ranks, oversample, seed, dtype=api.F64, variant=api.VARIANT_TTNN,
                 flags=0):
        self.tree, self.dims = tree, list(dims)
        self.plan = api.ttnn_plan_create(tree, dims, ranks, oversample, seed, variant=variant,
                                         sketch_dtype=dtype, flags=flags)
        self.state = api.ttnn_state_create(self.plan)
        self.sizes = api.ttnn_plan_sizes(self.plan)
        self.nodes = [api.ttnn_plan_node(self.plan, v) for v in range(len(tree[0]))]
        self.dtype = dtype

    def close(self):
        api.ttnn_state_destroy(self.state)
        api.ttnn_plan_destroy(self.plan)

    def state_host(self):
        import torch
        torch.cuda.synchronize()
        n, eb = self.sizes[0], self.sizes[1]
        buf = np.zeros(n, dtype=np.float64 if eb == 8 else np.float32)
        api.ttnn_state_save(self.state, buf)
        return buf.astype(np.float64)

    def sketches(self):
        """(Omega, Psi, Psi_root) dicts keyed by user node, like the oracle."""
        buf = self.state_host()
        Om, Ps, Pr = {}, {}, None
        for nd in self.nodes:
            if nd["parent"] < 0:
                Pr = buf[nd["psi_offset"]:nd["psi_offset"] + nd["psi_elems"]].reshape(nd["psi_shape"])
                continue
            if nd["identity"]:
                continue
            Om[nd["user_index"]] = buf[nd["omega_offset"]:nd["omega_offset"] + nd["omega_elems"]].reshape(nd["s"], nd["r"])
            Ps[nd["user_index"]] = buf[nd["psi_offset"]:nd["psi_offset"] + nd["psi_elems"]].reshape(nd["psi_shape"])
        return Om, Ps, Pr

    def recover(self):
        import torch
        core = torch.zeros(self.sizes[2], dtype=torch.float64, device="cuda")
        api.ttnn_recover(self.state, core)
        host = core.cpu().numpy()
        self.nodes = [api.ttnn_plan_node(self.plan, v) for v in range(len(self.tree[0]))]
        return {nd["user_index"]: host[nd["core_offset"]:nd["core_offset"] + nd["core_elems"]].reshape(nd["core_shape"])
                for nd in self.nodes}


def rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
