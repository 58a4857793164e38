def paper_mteps(V, E, n_src, seconds):
    return (V - 1) * E * n_src / seconds / 1e6
