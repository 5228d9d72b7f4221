"""Multi-box (batched) and served (queue) bindings -- declared when present."""


def declare(L):
    return L
