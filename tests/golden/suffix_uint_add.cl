__kernel void uadd(int x, int y, __global int *data)
{
    data[get_local_id(0)] = (int)((uint)y + (uint)x);
}
